// Internal definitions shared by the CUDA translation units of libagg.so.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "agg.h"

namespace agg {

// ---------------------------------------------------------------- geometry
constexpr int THREADS = 512;               // threads per block of the hash kernel
constexpr int RPT = 4;                     // rows per thread per tile
constexpr int TILE = THREADS * RPT;        // rows per block tile
constexpr uint32_t CH = 2048;              // records per staging chunk (32 KiB)
constexpr int MAX_FAN = 256;               // largest spill fan-out
constexpr uint32_t BUCKET = 32;            // slots per bucket: one 32-byte sector of tag bytes
constexpr uint32_t MIN_SLOTS = 4096;       // smallest active table of a round
constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr int64_t EMPTY_KEY = INT64_MIN;   // empty key slot; this one key value lives in a side slot
constexpr int64_t SKEY_EMPTY = INT64_MIN;  // empty marker of the shared-memory cache
constexpr int PHASES = 12;                 // phase timers kept by block 0
constexpr uint32_t NSUB_MAX = 4096;        // sub-partitions of one shared-memory round
#ifndef AGG_ROUND_CAP_M
#define AGG_ROUND_CAP_M 8
#endif
#ifndef AGG_GTABLE_DIV
#define AGG_GTABLE_DIV 2
#endif
constexpr uint64_t ROUND_CAP_MAX = (uint64_t)AGG_ROUND_CAP_M << 20;  // records of one shared-memory round
#ifndef AGG_ROUND_PACK_M
#define AGG_ROUND_PACK_M 4
#endif
// Partitions are packed into one round only up to this many records: a round
// this small stays in L2 from its count pass to its aggregate pass.  A single
// partition up to ROUND_CAP_MAX still gets a round of its own.
constexpr uint64_t ROUND_PACK_MAX = (uint64_t)AGG_ROUND_PACK_M << 20;
// At recursion levels >= 1 the global table (keys that overflow a block's
// shared-memory table, partitions too large for a shared-memory round) keeps
// 1/GTABLE_DIV of the slots; the rest of the entry memory is round scratch.
constexpr uint32_t GTABLE_DIV = AGG_GTABLE_DIV;
constexpr uint64_t REC_BYTES = 16;         // spilled record: (int64 key, int64 value)
constexpr int MAX_GRID = 1024;             // most blocks of one team (the sorted-input path counts per block)
// One tile adds at most TILE rows to a partition, so at most one new chunk is
// opened per partition per tile.
static_assert(TILE == (int)CH, "a tile is one staging chunk");

// Table entry layouts (bytes): key, count, sum, then MIN/MAX when requested.
enum EntKind { ENT32_CS = 0, ENT32_CSMM32 = 1, ENT64 = 2 };
inline __host__ __device__ uint32_t entry_bytes(int kind) { return kind == ENT64 ? 64u : 32u; }

// Control block at the start of the working memory (inside the budget).
// Fields under "run" are zeroed by the last block of every run; the barrier
// words persist.
struct alignas(128) Ctrl {
  unsigned int bar_count;
  unsigned int pad0[31];
  unsigned int bar_gen;
  unsigned int pad1[31];
  unsigned int done_count;
  unsigned int pad2[31];
  // ---- run
  unsigned long long status_bits;  // 1 << agg_status (cleared by agg_sync)
  unsigned long long occupancy;    // slots claimed in the current round
  unsigned long long out_count;    // groups written so far
  unsigned long long pool_next[2]; // chunks handed out per staging area
  unsigned long long rows_at_full; // level-0 row index of the first tile that spilled
  unsigned long long tile_next;    // level-0 tiles claimed so far (dynamic tile assignment)
  unsigned long long rounds;
  unsigned long long phase_ns[PHASES];
  unsigned long long spill_records[AGG_MAX_LEVELS];
  unsigned long long resident_groups[AGG_MAX_LEVELS];
  unsigned long long part_records[2][MAX_FAN];
  unsigned int part_chunks[2][MAX_FAN];
  unsigned int part_cursor[2][MAX_FAN];
  // shared-memory rounds of levels >= 1 (two sets by round parity)
  unsigned int sub_tot[2][NSUB_MAX];       // records per sub-partition (column totals of the scan)
  unsigned int sub_base[2][NSUB_MAX + 1];  // start of each sub-partition in the scratch
  unsigned long long lvl_sub_records[2];  // records aggregated in shared memory (by round parity)
  unsigned long long lvl_sub_groups[2];   // groups they formed (keys-per-record estimate)
  unsigned int overflow_used[2];          // a key of the level (by parity) went to the global table
  unsigned int sub_next[2];               // pass C: sub-partitions claimed so far (by round parity)
  unsigned int sorted_fail;               // sorted-input path: a key below its predecessor was found
  unsigned int sorted_used;               // sorted-input path: this run completed on it
  unsigned long long sorted_heads[MAX_GRID];  // sorted-input path: segment heads in each block's rows
  unsigned int fallback_now;              // this level's records go to the sort fallback
  unsigned int ovf_listed;                // in-budget partitions: overflow-table slots claimed (listed)
  unsigned long long fallback_records;    // records aggregated by the sort fallback
  unsigned long long fallback_level;      // level at which it ran (0 = none)
  // ---- snapshot of the last completed run
  unsigned long long last_n_rows;
  unsigned long long last_n_groups;
  unsigned long long last_levels;
  unsigned long long last_rounds;
  unsigned long long last_rows_at_full;
  unsigned long long last_phase_ns[PHASES];
  unsigned long long last_spill_records[AGG_MAX_LEVELS];
  unsigned long long last_resident_groups[AGG_MAX_LEVELS];
  unsigned long long last_sorted;         // 1 when the last run took the sorted-input path
  unsigned long long last_fallback_records;
  unsigned long long last_fallback_level;
};

// Everything one hash-path kernel launch needs (passed by value).
struct HashParams {
  const int64_t* keys;
  const void* vals;
  uint64_t n;
  int vec_ok;          // keys/vals aligned for vector loads
  int has_vals;
  int64_t* o_keys;
  uint64_t* o_count;
  int64_t* o_sum;
  int64_t* o_min;
  int64_t* o_max;
  uint64_t o_cap;
  uint64_t* o_ngroups;
  Ctrl* ctrl;
  uint8_t* ent;
  uint32_t* tags;
  uint32_t slots;      // physical slots S (multiple of BUCKET); entry `slots` is the side slot
  uint8_t* stg[2];     // staging areas (chunks of CH records)
  uint32_t* dir_part[2];
  uint32_t* dir_count[2];
  uint32_t* list[2];
  uint64_t max_chunks[2];
  uint64_t seed;
  uint32_t ops;
  uint32_t fan_log2;
  double lf;           // maximum load factor
  uint32_t s_act0;     // active slots at level 0
  uint32_t ns;         // shared-memory table entries (power of two)
  uint32_t dedup;      // warp-level key dedup on/off
  uint32_t cache;      // shared-memory cache of resident groups on/off
  uint32_t no_prefetch;  // input in host memory: no bulk L2 prefetch of input tiles
  uint32_t sorted_probe; // try the sorted-input path first (a sampled order check decides)
  uint32_t max_levels;   // records reaching this level go to the sort fallback
  uint32_t fallback_ok;  // the sort fallback has its shared memory and scratch (else the depth cap is an error)
  uint32_t stg_host;     // the staging areas are in host memory (reached over the host link)
  uint64_t timeout_ns; // bounded waits give up after this long
};

struct KernelInfo {
  int blocks;          // cooperative grid size
  size_t smem;         // dynamic shared memory per block
};

// hash_path.cu
// Depth cap and availability of the sort fallback for a run of `blocks` blocks
// over `slots` table slots of `es` bytes with `ns` shared-memory entries
// (`max_levels` 0 = default: the levels a sort-based algorithm would need).
void hash_fallback_plan(uint32_t fan, uint32_t max_levels, uint32_t blocks, uint64_t slots, uint32_t es, uint32_t ns,
                        bool staging, HashParams* p);
cudaError_t hash_kernel_info(int ent_kind, int vt, uint32_t ns, int device, KernelInfo* out);
cudaError_t hash_launch(int ent_kind, int vt, const HashParams& p, const KernelInfo& ki, cudaStream_t s);
cudaError_t hash_init_table(uint8_t* ent, uint32_t* tags, uint32_t slots, int ent_kind, cudaStream_t s);
// In-budget fast path: the active slots for n rows, or 0 when n rows may not fit
// (more than half the slots); then two ordinary launches (aggregate, emit).
uint32_t hash_fast_slots(uint64_t n, uint64_t slots);
cudaError_t hash_fast_launch(int ent_kind, int vt, const HashParams& p, uint32_t s_act, size_t smem, cudaStream_t s);
// Partitioned in-budget path for small inputs (no global atomics): the plan
// (false when n rows are too many, or the scratch and overflow table do not fit
// the slots), then two launches (partition, aggregate + emit).  The scratch
// occupies the entries from scratch_slot up to the side slot, which are left
// dirty: the caller restores them before another path uses the table.
struct PartPlan {
  uint32_t nblk = 0;          // first-launch blocks (FAST rows each)
  uint32_t plog = 0;          // log2 of the partitions
  uint32_t s_ovf = 0;         // slots of the overflow table [0, s_ovf)
  uint32_t scratch_slot = 0;  // first entry used as scratch
};
// Resets `count` table entries starting at ent to the empty state (tags untouched).
cudaError_t hash_reset_entries(uint8_t* ent, uint64_t count, int ent_kind, cudaStream_t s);
bool hash_part_plan(uint64_t n, uint64_t slots, uint32_t es, uint32_t ns, PartPlan* out);
cudaError_t hash_part_launch(int ent_kind, int vt, const HashParams& p, const PartPlan& pp, uint32_t es, size_t smem,
                             cudaStream_t s);
cudaError_t hash_batch_kernel_info(int ent_kind, int vt, uint32_t ns, int device, KernelInfo* out);
cudaError_t hash_batch_launch(int ent_kind, int vt, const HashParams* items, const uint32_t* team_off,
                              const uint32_t* team_items, uint32_t team_blocks, uint32_t nteams, size_t smem,
                              cudaStream_t s);

}  // namespace agg
