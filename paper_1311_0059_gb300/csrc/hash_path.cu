// Hash path of the budgeted group-by: one persistent cooperative kernel per run.
//
// Level 0 streams the input once (Section 4.3, Phase 1), in tiles claimed
// dynamically by the blocks.  Each row's key is hashed once with the
// MurmurHash3 64-bit finaliser under a per-level seed (Section 6.7).  A
// per-block, 4-way set-associative shared-memory cache of resident groups
// absorbs hot keys (optionally after combining equal keys inside a warp), and
// the remaining updates go to the global open-addressing table with 64-bit
// atomics.  The table follows the Pre-Partitioning policy (Section 4.3.4):
// every group that finds room in the table before the table is full is
// resident and completes in place; a group that finds no room is spilled, and
// it is spilled whole.  Spilled rows are radix-partitioned on hash bits into
// staging chunks (the run files of Section 4.3), ranked by shared-memory
// atomics.  After the pass the table is emitted and reset.  Spilled partitions
// are then processed level by level (Phase 2) with fresh seeds; partitions are
// packed into rounds (partition tuning, Section 4.3.3), and each round is
// split into sub-partitions that one block aggregates in shared memory.
// Phases are separated by grid barriers whose waits are bounded.
//
// Table and residency.  Slots form buckets of 32; a key may live only in its
// hash bucket, in the first slot of its own probe order (a rotation chosen by
// hash bits) that was free when it arrived.  A key slot changes once per
// round, from EMPTY to a key, by a 64-bit atomicCAS, so "k is absent and its
// bucket holds 32 other keys" can never become false later in the round: such
// a key spills consistently, and a key is never both resident and spilled.
// "Full" (Section 3.2: no new group fits) is therefore judged per bucket.  A
// tag byte per slot (8 hash bits, never zero, written after the claim) is a
// compact filter kept in L2: a probe reads its bucket's 32 tags in one 32-byte
// sector and reads keys only where a tag matches or is still zero.  The key
// value that marks an empty slot (INT64_MIN) is kept in a dedicated side slot.
#include <cstdio>

#include "agg_internal.cuh"

namespace agg {
namespace {

constexpr unsigned FULL_MASK = 0xFFFFFFFFu;
constexpr int WARPS = THREADS / 32;
constexpr uint32_t TLIST = 128;  // tiles of a round pass whose chunk ids are staged at once
constexpr uint32_t A_TILES = 4;  // tiles whose keys one step of the count pass loads together

__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// Seed of recursion level L: a fresh, uncorrelated hash function per level.
__device__ __forceinline__ uint64_t level_seed(uint64_t seed, uint32_t level) {
  return fmix64(seed + 0xD6E8FEB86659FD93ull * (uint64_t)(level + 1));
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Asks the memory system to stage [p, p + bytes) in L2 (p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  if (bytes >= 16) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes & ~15u) : "memory");
}

__device__ __forceinline__ void set_status(Ctrl* c, agg_status s) {
  atomicOr(&c->status_bits, 1ull << (int)s);
}


// Adds v to a 64-bit word in shared memory, exactly modulo 2^64, with 32-bit
// atomics: the low word takes the low half of v and reports the carry it
// produced; the high word takes the high half plus that carry (skipped when
// zero, the common case for small values).  64-bit shared-memory additions
// have no native atomic and contend badly on hot words.
// Shared-memory accesses of the partial-state tables, in the shared state
// space explicitly (the tables are reached through pointers, and a generic
// atomic on shared memory is far slower than a shared one).
__device__ __forceinline__ uint32_t sh_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ long long sh_cas_s64(long long* p, long long cmp, long long val) {
  long long old;
  asm volatile("atom.shared.cas.b64 %0, [%1], %2, %3;" : "=l"(old) : "r"(sh_addr(p)), "l"(cmp), "l"(val) : "memory");
  return old;
}

__device__ __forceinline__ uint32_t sh_atom_add_u32(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(sh_addr(p)), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void sh_red_add_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(sh_addr(p)), "r"(v) : "memory");
}

__device__ __forceinline__ void sh_red_min_s64(long long* p, long long v) {
  asm volatile("red.shared.min.s64 [%0], %1;" ::"r"(sh_addr(p)), "l"(v) : "memory");
}

__device__ __forceinline__ void sh_red_max_s64(long long* p, long long v) {
  asm volatile("red.shared.max.s64 [%0], %1;" ::"r"(sh_addr(p)), "l"(v) : "memory");
}

// MIN and MAX in shared memory only ever move one way, so an update that does
// not improve the value read first is a no-op and is skipped: a value at or
// above the minimum seen now is at or above the final minimum.  Most rows of a
// hot key then touch the word with a plain load instead of an atomic.
__device__ __forceinline__ long long sh_ld_volatile_s64(const long long* p) {
  long long v;
  asm volatile("ld.volatile.shared.s64 %0, [%1];" : "=l"(v) : "r"((uint32_t)__cvta_generic_to_shared(p)) : "memory");
  return v;
}

#ifndef AGG_PASSC_PREFETCH
#define AGG_PASSC_PREFETCH 1
#endif
#ifndef AGG_MINMAX_SKIP
#define AGG_MINMAX_SKIP 1
#endif
__device__ __forceinline__ void sh_min_s64(long long* p, long long v) {
  if (!AGG_MINMAX_SKIP || v < sh_ld_volatile_s64(p)) sh_red_min_s64(p, v);
}

__device__ __forceinline__ void sh_max_s64(long long* p, long long v) {
  if (!AGG_MINMAX_SKIP || v > sh_ld_volatile_s64(p)) sh_red_max_s64(p, v);
}

__device__ __forceinline__ void smem_add_u64(unsigned long long* p, unsigned long long v) {
  uint32_t* w = reinterpret_cast<uint32_t*>(p);
  const uint32_t lo = (uint32_t)v;
  const uint32_t old = sh_atom_add_u32(w, lo);
  const uint32_t inc = (uint32_t)(v >> 32) + ((uint32_t)(old + lo) < old ? 1u : 0u);
  if (inc) sh_red_add_u32(w + 1, inc);
}

// ---------------------------------------------------------------- shared memory

struct Smem {
  uint32_t cnt[MAX_FAN];   // spill: rows of this tile per partition; P1: chunk histogram
  uint32_t cur[MAX_FAN];   // current staging chunk per partition (NONE = none)
  uint32_t fill[MAX_FAN];  // records in the current chunk (CH when none)
  uint32_t nxt[MAX_FAN];   // chunk opened for this tile's overflow
  uint32_t pend[MAX_FAN];  // records of the last spilling tile not yet applied to cur/fill
  uint32_t begin[MAX_FAN + 1];
  unsigned long long hrec[MAX_FAN];
  unsigned long long pspill[MAX_FAN];  // rows spilled to each partition at this level (by its fan-loop thread)
  unsigned long long scan_base;
  uint32_t warp_tot[WARPS];
  uint32_t scan_total;
  uint32_t ok;
  uint32_t first_spill;
  uint32_t tiles;      // tiles processed by this block (adaptive sampling clock)
  uint32_t flush_tiles;  // tiles since the shared-memory cache was last flushed
  uint32_t use_cache;
  uint32_t use_dedup;
  uint32_t st_rows, st_hits, st_dups;
  unsigned long long tile_q[2];  // level-0 tiles claimed by this block (current, next) by iteration parity
  uint32_t sub_q[2];            // pass C: sub-partitions claimed by this block, by iteration parity
  uint32_t tl_chunk[TLIST];     // staged tiles of a round pass: chunk id
  uint32_t tl_count[TLIST];     // and its record count
  // sorted-input path: per-warp totals of a segmented scan, the carry into the
  // next tile, and the block's leading partial segment
  unsigned long long sw_c[WARPS], sw_s[WARPS];
  long long sw_mn[WARPS], sw_mx[WARPS];
  uint32_t sw_f[WARPS];
  unsigned long long tc_c, tc_s;
  long long tc_mn, tc_mx;
  uint32_t tc_f;
  unsigned long long lead_c, lead_s;
  long long lead_mn, lead_mx;
  uint32_t lead_valid;
  uint32_t vote;
  // segmented scan: carry into each warp, head counts, warp-edge keys
  unsigned long long wc_c[WARPS], wc_s[WARPS];
  long long wc_mn[WARPS], wc_mx[WARPS];
  uint32_t wc_f[WARPS];
  uint32_t wh[WARPS + 1];
  long long wl_key[WARPS], wf_key[WARPS];
  long long tile_prev_key;
  // the level at which run_groupby handed its records to the sort fallback
  unsigned long long fb_nch;
  uint32_t fb_level, fb_src, fb_dst, fb_set;
};

// Shared-memory table of partial states.  Counts are 32-bit (an entry is
// flushed before it can see 2^31 rows); sums are 64-bit words updated with
// smem_add_u64; MIN/MAX use the native 64-bit atomics.
struct Cache {
  long long* key;
  unsigned long long* sum;
  long long* mn;
  long long* mx;
  unsigned* cnt;
  uint32_t* slot;
  uint32_t n;  // 0 = disabled
};

__host__ __device__ inline size_t cache_bytes(uint32_t ns, bool mm) {
  return (size_t)ns * (8 + 8 + 4 + 4 + (mm ? 16 : 0));
}

__device__ inline Cache carve_cache(unsigned char* base, uint32_t ns, bool mm) {
  Cache c;
  c.n = ns;
  unsigned char* p = base;
  c.key = reinterpret_cast<long long*>(p);
  p += (size_t)ns * 8;
  c.sum = reinterpret_cast<unsigned long long*>(p);
  p += (size_t)ns * 8;
  if (mm) {
    c.mn = reinterpret_cast<long long*>(p);
    p += (size_t)ns * 8;
    c.mx = reinterpret_cast<long long*>(p);
    p += (size_t)ns * 8;
  } else {
    c.mn = c.mx = nullptr;
  }
  c.cnt = reinterpret_cast<unsigned*>(p);
  p += (size_t)ns * 4;
  c.slot = reinterpret_cast<uint32_t*>(p);
  return c;
}

// ---------------------------------------------------------------- grid barrier

// The blocks that run one group-by together: the whole grid for agg_run, a
// slice of it for one instance of a batch.  nb == 1 makes every team barrier a
// __syncthreads.
struct Team {
  uint32_t nb;   // blocks in the team
  uint32_t bid;  // this block's index in the team
};

// Counting barrier over the team's blocks (co-resident: cooperative launch).
// The wait is bounded: after timeout_ns the block records AGG_ERR_TIMEOUT and
// returns false.
__device__ bool grid_barrier(const Team& T, Ctrl* c, uint64_t timeout_ns, Smem& S) {
  if (T.nb == 1) {
    __syncthreads();
    return true;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t ok = 1;
    const uint32_t g = ld_acquire_u32(&c->bar_gen);
    __threadfence();
    const uint32_t arrived = atomicAdd(&c->bar_count, 1u) + 1u;
    if (arrived == T.nb) {
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      const uint64_t t0 = globaltimer();
      while (ld_acquire_u32(&c->bar_gen) == g) {
        __nanosleep(32);
        if (globaltimer() - t0 > timeout_ns) {
          set_status(c, AGG_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    S.ok = ok;
  }
  __syncthreads();
  return S.ok != 0;
}

// Phase indices of Ctrl::phase_ns (block 0's view).
enum Phase { PH_L0 = 0, PH_L0_WAIT, PH_L0_EMIT, PH_LISTS, PH_ROUND_AGG, PH_ROUND_WAIT, PH_ROUND_EMIT, PH_TOTAL,
             PH_SUB_COUNT, PH_SUB_SCATTER, PH_SUB_AGG };

// Phase timer of block 0 (diagnostics, reported by agg_get_stats).
struct Timer {
  uint64_t t;
  __device__ void start(const Team& T) {
    if (T.bid == 0 && threadIdx.x == 0) t = globaltimer();
  }
  __device__ void lap(const Team& T, Ctrl* c, int phase) {
    if (T.bid == 0 && threadIdx.x == 0) {
      const uint64_t now = globaltimer();
      c->phase_ns[phase] += now - t;
      t = now;
    }
  }
};

// ---------------------------------------------------------------- table access

template <int ENT>
struct Ent {
  static constexpr uint32_t ES = ENT == ENT64 ? 64u : 32u;
  static constexpr bool MM = ENT != ENT32_CS;
  __device__ static uint8_t* at(uint8_t* base, uint32_t slot) { return base + (size_t)slot * ES; }
  __device__ static void add(uint8_t* e, uint32_t ops, unsigned long long c, unsigned long long s, long long mn,
                             long long mx) {
    if (ops & AGG_COUNT) atomicAdd(reinterpret_cast<unsigned long long*>(e + 8), c);
    if (ops & AGG_SUM) atomicAdd(reinterpret_cast<unsigned long long*>(e + 16), s);
    if (ENT == ENT32_CSMM32) {
      if (ops & AGG_MIN) atomicMin(reinterpret_cast<int*>(e + 24), (int)mn);
      if (ops & AGG_MAX) atomicMax(reinterpret_cast<int*>(e + 28), (int)mx);
    } else if (ENT == ENT64) {
      if (ops & AGG_MIN) atomicMin(reinterpret_cast<long long*>(e + 24), mn);
      if (ops & AGG_MAX) atomicMax(reinterpret_cast<long long*>(e + 32), mx);
    }
  }
  __device__ static void reset(uint8_t* e) {
    __stcg(reinterpret_cast<long long*>(e), (long long)EMPTY_KEY);
    __stcg(reinterpret_cast<unsigned long long*>(e + 8), 0ull);
    __stcg(reinterpret_cast<unsigned long long*>(e + 16), 0ull);
    if (ENT == ENT32_CSMM32) {
      __stcg(reinterpret_cast<int*>(e + 24), INT32_MAX);
      __stcg(reinterpret_cast<int*>(e + 28), INT32_MIN);
    } else if (ENT == ENT64) {
      __stcg(reinterpret_cast<long long*>(e + 24), (long long)INT64_MAX);
      __stcg(reinterpret_cast<long long*>(e + 32), (long long)INT64_MIN);
    }
  }
  __device__ static void read(uint8_t* e, long long& key, unsigned long long& c, unsigned long long& s, long long& mn,
                              long long& mx) {
    key = __ldcg(reinterpret_cast<const long long*>(e));
    c = __ldcg(reinterpret_cast<const unsigned long long*>(e + 8));
    s = __ldcg(reinterpret_cast<const unsigned long long*>(e + 16));
    if (ENT == ENT32_CSMM32) {
      mn = __ldcg(reinterpret_cast<const int*>(e + 24));
      mx = __ldcg(reinterpret_cast<const int*>(e + 28));
    } else if (ENT == ENT64) {
      mn = __ldcg(reinterpret_cast<const long long*>(e + 24));
      mx = __ldcg(reinterpret_cast<const long long*>(e + 32));
    } else {
      mn = mx = 0;
    }
  }
};

// Candidate slots of a bucket: tag byte equal to the key's tag, or still zero
// (free, or claimed a moment ago with its tag not yet written).  The bucket's
// 32 tag bytes are one 32-byte sector, read with one 256-bit load and tested
// four bytes at a time with an exact zero-byte test: bit 7 of each byte of
// ((v & 0x7F..) + 0x7F..) | v is set iff that byte of v is non-zero.  The mask
// is built in word-interleaved order (bit 8b + i stands for byte b of tag word
// i, slot cand_slot(8b + i) = 4i + b), which needs no gathering of bits; the
// probe order only has to be fixed per key, not ascending.
__device__ __forceinline__ uint32_t bucket_candidates(const HashParams& P, uint32_t b, uint32_t tag4) {
  unsigned long long q0, q1, q2, q3;
  asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];"
               : "=l"(q0), "=l"(q1), "=l"(q2), "=l"(q3)
               : "l"(reinterpret_cast<const uint8_t*>(P.tags) + (size_t)b * BUCKET));
  const unsigned long long q[4] = {q0, q1, q2, q3};
  uint32_t cand = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t w = (i & 1) ? (uint32_t)(q[i >> 1] >> 32) : (uint32_t)q[i >> 1];
    const uint32_t x = w ^ tag4;
    const uint32_t nz_x = ((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x;
    const uint32_t nz_w = ((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w;
    cand |= (~(nz_x & nz_w) & 0x80808080u) >> (7 - i);
  }
  return cand;
}

// Slot within its bucket of candidate bit p (see bucket_candidates).
__device__ __forceinline__ uint32_t cand_slot(uint32_t p) { return 4 * (p & 7) + (p >> 3); }

__device__ __forceinline__ uint32_t home_bucket(uint64_t h, uint32_t s_act) {
  return (uint32_t)(((h >> 32) * (uint64_t)(s_act / BUCKET)) >> 32);
}

// Tag byte of a key: 8 hash bits, 1..255 (0 marks a free slot).
__device__ __forceinline__ uint32_t key_tag(uint64_t h) {
  const uint32_t t = (uint32_t)(h & 0xFFu);
  return t ? t : 1u;
}

// First slot of a key's probe order inside its bucket (hash bits 27..31).  Each
// key walks the bucket from its own starting slot, wrapping around, so that
// concurrent inserts of different keys do not all race for slot 0.
__device__ __forceinline__ uint32_t key_start(uint64_t h) { return (uint32_t)(h >> 27) & (BUCKET - 1); }

// Candidate mask in a key's probe order: bit j stands for candidate position
// (start + j) mod 32, that is slot cand_slot((start + j) mod 32).
__device__ __forceinline__ uint32_t rotate_cand(uint32_t cand, uint32_t start) {
  return __funnelshift_r(cand, cand, start);
}

// Finds or claims the slot of `key` in its bucket, given the bucket's candidate
// mask in the key's probe order (`cand`, see rotate_cand) and the key word of
// its first candidate slot (`k_first`, loaded by the caller so that the loads
// of several rows overlap).  A key may live only in its bucket, in the first
// slot of its probe order that was free when it arrived: the candidates are
// visited in that order; a free slot is claimed by a 64-bit CAS; a slot taken
// meanwhile by another key is passed.  Every insert of the same key walks the
// same order, so a key is never claimed twice.  Returns the slot when the key
// is (now) resident, -1 when the bucket holds 32 other keys (the key spills).
// *claimed is set when this call inserted it.
template <int ENT>
__device__ long long probe_table(const HashParams& P, uint32_t b, uint32_t cand, uint32_t start, long long key,
                                 uint32_t tag, uint32_t& claimed, long long k_first) {
  if (key == EMPTY_KEY) {  // the empty marker value itself: side slot, always resident
    uint8_t* tb = reinterpret_cast<uint8_t*>(P.tags) + P.slots;
    if (__ldcg(tb) == 0) __stcg(tb, (uint8_t)0x80);
    return P.slots;
  }
  bool first = true;
  while (cand) {
    const uint32_t i = cand_slot((__ffs(cand) - 1 + start) & (BUCKET - 1));
    cand &= cand - 1;
    const uint32_t slot = b * BUCKET + i;
    long long* kp = reinterpret_cast<long long*>(Ent<ENT>::at(P.ent, slot));
    const long long k2 = first ? k_first : __ldcg(kp);
    first = false;
    if (k2 == key) return slot;
    if (k2 != EMPTY_KEY) continue;
    const long long old = (long long)atomicCAS(reinterpret_cast<unsigned long long*>(kp),
                                               (unsigned long long)EMPTY_KEY, (unsigned long long)key);
    if (old == EMPTY_KEY) {
      __stcg(reinterpret_cast<uint8_t*>(P.tags) + slot, (uint8_t)tag);
      claimed = 1;
      return slot;
    }
    if (old == key) return slot;
  }
  return -1;
}

// ---------------------------------------------------------------- per-level context

struct Level {
  uint32_t level;
  uint64_t seed;
  uint32_t s_act;     // active slots of this round (multiple of BUCKET)
  uint32_t dst;       // staging area receiving this level's spills
  uint32_t fan_mask;
};

// The level-0 cache is 4-way set associative: a key may occupy only the four
// entries of its set (n / 4 sets), so a probe is one 32-byte read and four
// compares, with no probe loop for the warp to wait on.
constexpr uint32_t CACHE_WAYS = 4;

__device__ __forceinline__ uint32_t cache_set(const Cache& cc, uint64_t h) {
  return ((uint32_t)(h >> 16) & (cc.n / CACHE_WAYS - 1)) * CACHE_WAYS;
}

__device__ __forceinline__ void sh_ld_volatile_s64x2(const long long* p, long long& a, long long& b) {
  asm volatile("ld.volatile.shared.v2.s64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(sh_addr(p)) : "memory");
}

// Shared-memory cache probe; true when the key's partial state was updated.
// *free_way tells whether the set had a free way (worth an insert later).
template <int ENT>
__device__ __forceinline__ bool cache_hit(const Cache& cc, long long key, uint64_t h, unsigned long long c,
                                          unsigned long long s, long long mn, long long mx, bool& free_way) {
  free_way = false;
  if (cc.n == 0 || key == SKEY_EMPTY) return false;
  const uint32_t b = cache_set(cc, h);
  long long k0, k1, k2, k3;
  sh_ld_volatile_s64x2(cc.key + b, k0, k1);
  sh_ld_volatile_s64x2(cc.key + b + 2, k2, k3);
  const int way = k0 == key ? 0 : k1 == key ? 1 : k2 == key ? 2 : k3 == key ? 3 : -1;
  if (way < 0) {
    free_way = k0 == SKEY_EMPTY || k1 == SKEY_EMPTY || k2 == SKEY_EMPTY || k3 == SKEY_EMPTY;
    return false;
  }
  const uint32_t idx = b + (uint32_t)way;
  sh_red_add_u32(cc.cnt + idx, (uint32_t)c);
  smem_add_u64(cc.sum + idx, s);
  if (Ent<ENT>::MM) {
    sh_min_s64(cc.mn + idx, mn);
    sh_max_s64(cc.mx + idx, mx);
  }
  return true;
}

// Records a resident key's global slot in a free way of its cache set (first
// come, first kept; entries are never evicted before a flush).
__device__ __forceinline__ void cache_insert(const Cache& cc, Smem& S, long long key, uint64_t h, uint32_t slot) {
  if (cc.n == 0 || key == SKEY_EMPTY) return;
  const uint32_t b = cache_set(cc, h);
#pragma unroll
  for (uint32_t w = 0; w < CACHE_WAYS; ++w) {
    const long long old = sh_cas_s64(cc.key + b + w, SKEY_EMPTY, key);
    if (old == SKEY_EMPTY) {
      cc.slot[b + w] = slot;
      return;
    }
    if (old == key) return;
  }
}

template <int ENT>
__device__ void cache_flush(const HashParams& P, const Cache& cc, Smem& S) {
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < cc.n; i += THREADS) {
    const long long k = cc.key[i];
    if (k == SKEY_EMPTY) continue;
    const unsigned long long c = cc.cnt[i];
    if (c) {
      Ent<ENT>::add(Ent<ENT>::at(P.ent, cc.slot[i]), P.ops, c, cc.sum[i], Ent<ENT>::MM ? cc.mn[i] : 0,
                    Ent<ENT>::MM ? cc.mx[i] : 0);
    }
    cc.key[i] = SKEY_EMPTY;
    cc.cnt[i] = 0;
    cc.sum[i] = 0;
    if (Ent<ENT>::MM) {
      cc.mn[i] = INT64_MAX;
      cc.mx[i] = INT64_MIN;
    }
  }
  if (threadIdx.x == 0) S.flush_tiles = 0;
  __syncthreads();
}

// A cache entry counts in 32 bits: flushing at least every 2^20 tiles (2^31
// rows of one block) keeps every count below 2^32.
constexpr uint32_t CACHE_FLUSH_TILES = 1u << 20;

// ---------------------------------------------------------------- one tile of rows

// Per-block adaptive features: every SAMPLE_PERIOD tiles, SAMPLE_TILES tiles
// run with warp dedup and the shared-memory cache both on and count how many
// rows each saves; the block keeps a feature on while it pays.
constexpr uint32_t SAMPLE_PERIOD = 128, SAMPLE_TILES = 2;

__device__ __forceinline__ void adapt_begin_tile(Smem& S, bool cache_allowed, bool dedup_allowed) {
  if (threadIdx.x == 0) {
    const bool sampling = (S.tiles % SAMPLE_PERIOD) < SAMPLE_TILES;
    if (sampling) {
      S.use_cache = cache_allowed;
      S.use_dedup = dedup_allowed;
    }
  }
}

__device__ __forceinline__ void adapt_end_tile(Smem& S, bool cache_allowed, bool dedup_allowed) {
  if (threadIdx.x == 0) {
    const uint32_t ph = S.tiles % SAMPLE_PERIOD;
    if (ph == SAMPLE_TILES - 1) {
      const uint32_t rows = S.st_rows ? S.st_rows : 1;
      S.use_cache = cache_allowed && S.st_hits * 20u >= rows;   // >= 5% of rows absorbed
      S.use_dedup = dedup_allowed && S.st_dups * 50u >= rows;   // >= 2% of rows combined
      S.st_rows = S.st_hits = S.st_dups = 0;
    }
    S.tiles += 1;
    S.flush_tiles += 1;
  }
}

template <int ENT>
__device__ void global_and_spill(const HashParams& P, const Level& L, Smem& S, const Cache& cc, long long (&k)[RPT],
                                 long long (&v)[RPT], const uint64_t (&h)[RPT], const bool (&need)[RPT],
                                 const bool (&cfree)[RPT], uint64_t tile_row0, bool cache_ins);

// Aggregates up to RPT rows per thread (block-uniform call), then spills the
// rows whose keys are not resident.  `tile_row0` orders level-0 tiles.
template <int ENT>
__device__ void process_rows(const HashParams& P, const Level& L, Smem& S, const Cache& cc, long long (&k)[RPT],
                             long long (&v)[RPT], bool (&valid)[RPT], uint64_t tile_row0) {
  const uint32_t lane = threadIdx.x & 31;
  const bool use_cache = S.use_cache && cc.n;
  const bool use_dedup = S.use_dedup;
  const bool sampling = (S.tiles % SAMPLE_PERIOD) < SAMPLE_TILES;
  bool need[RPT];
  bool cfree[RPT];  // the row's cache set had a free way when probed (or was not probed)
  uint64_t h[RPT];  // each row's hash under this level's seed, computed once
  uint32_t hits = 0, dups = 0;

  // ---- shared-memory cache of resident groups (with warp dedup of equal keys)
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    need[r] = valid[r];
    cfree[r] = true;
    h[r] = fmix64((uint64_t)k[r] ^ L.seed);
  }
  if (use_cache) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const bool val = valid[r];
      uint32_t peers = 1u << lane, leader = lane;
      unsigned long long gc = 1, gs = (unsigned long long)v[r];
      long long gmn = v[r], gmx = v[r];
      if (use_dedup) {
        const uint32_t vm = __ballot_sync(FULL_MASK, val);
        if (val) peers = __match_any_sync(vm, k[r]);
        leader = __ffs(peers) - 1;
        const uint32_t gsize = __popc(peers);
        const uint32_t maxg = __reduce_max_sync(FULL_MASK, gsize);
        if (maxg > 1) {
          uint32_t rem = (val && lane == leader) ? (peers & ~(1u << lane)) : 0u;
          for (uint32_t it = 1; it < maxg; ++it) {
            const int src = rem ? __ffs(rem) - 1 : (int)lane;
            rem &= rem - 1;
            const long long ov = __shfl_sync(FULL_MASK, v[r], src);
            if (src != (int)lane) {
              gs += (unsigned long long)ov;
              if (Ent<ENT>::MM) {
                gmn = ov < gmn ? ov : gmn;
                gmx = ov > gmx ? ov : gmx;
              }
            }
          }
          gc = gsize;
        }
        if (sampling && val && lane == leader) dups += gsize - 1;
      }
      bool hit = false, cf = true;
      if (val && lane == leader) {
        hit = cache_hit<ENT>(cc, k[r], h[r], gc, gs, gmn, gmx, cf);
        if (sampling) hits += hit ? (uint32_t)gc : 0u;
      }
      if (use_dedup) {
        hit = __shfl_sync(FULL_MASK, hit, leader);
        cf = __shfl_sync(FULL_MASK, cf, leader);
      }
      need[r] = val && !hit;
      cfree[r] = cf;
    }
  } else if (sampling && use_dedup) {
    // no cache: dedup only measured (global updates stay per row)
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const uint32_t vm = __ballot_sync(FULL_MASK, valid[r]);
      if (valid[r]) {
        const uint32_t peers = __match_any_sync(vm, k[r]);
        if ((int)lane == __ffs(peers) - 1) dups += __popc(peers) - 1;
      }
    }
  }

  if (sampling) {
    uint32_t nv = 0;
#pragma unroll
    for (int r = 0; r < RPT; ++r) nv += valid[r];
    const uint32_t a = __reduce_add_sync(FULL_MASK, nv), b = __reduce_add_sync(FULL_MASK, hits),
                   c = __reduce_add_sync(FULL_MASK, dups);
    if (lane == 0) {
      atomicAdd(&S.st_rows, a);
      atomicAdd(&S.st_hits, b);
      atomicAdd(&S.st_dups, c);
    }
  }

  global_and_spill<ENT>(P, L, S, cc, k, v, h, need, cfree, tile_row0, use_cache || sampling);
}

// Updates the global table for every row with need[r] set (claiming slots for
// new keys), then spills the rows whose keys are not resident to the next
// level's partitions.  Block-uniform call.  `cache_ins` records newly found
// slots in the shared-memory cache.
template <int ENT>
__device__ void global_and_spill(const HashParams& P, const Level& L, Smem& S, const Cache& cc, long long (&k)[RPT],
                                 long long (&v)[RPT], const uint64_t (&h)[RPT], const bool (&need)[RPT],
                                 const bool (&cfree)[RPT], uint64_t tile_row0, bool cache_ins) {
  // ---- global table: bucket tags of every remaining row first, then resolve
  uint32_t cand[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    cand[r] = 0;
    if (need[r] && k[r] != EMPTY_KEY)
      cand[r] = rotate_cand(bucket_candidates(P, home_bucket(h[r], L.s_act), key_tag(h[r]) * 0x01010101u),
                            key_start(h[r]));
  }
  // key word of every row's first candidate slot, all loads in flight together
  long long kf[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    kf[r] = EMPTY_KEY;
    if (cand[r]) {
      const uint32_t slot =
          home_bucket(h[r], L.s_act) * BUCKET + cand_slot((__ffs(cand[r]) - 1 + key_start(h[r])) & (BUCKET - 1));
      kf[r] = __ldcg(reinterpret_cast<const long long*>(Ent<ENT>::at(P.ent, slot)));
    }
  }
  bool sp[RPT];
  bool any_sp = false;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    sp[r] = false;
    if (!need[r]) continue;
    uint32_t claimed = 0;
    const long long slot =
        probe_table<ENT>(P, home_bucket(h[r], L.s_act), cand[r], key_start(h[r]), k[r], key_tag(h[r]), claimed, kf[r]);
    if (slot >= 0) {
      Ent<ENT>::add(Ent<ENT>::at(P.ent, (uint32_t)slot), P.ops, 1ull, (unsigned long long)v[r], v[r], v[r]);
      if (cache_ins && cfree[r]) cache_insert(cc, S, k[r], h[r], (uint32_t)slot);
    } else {
      sp[r] = true;
      any_sp = true;
    }
  }

  // ---- spill: ranks per partition from one shared-memory atomic per row
  // (cheaper than warp aggregation with __match_any_sync), taken before the
  // block knows whether any row spills (a tile without spills adds nothing to
  // the counters), so that the vote below also serves as the barrier after them
  uint32_t part[RPT], rank[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    part[r] = (uint32_t)(h[r] >> 8) & L.fan_mask;
    rank[r] = sp[r] ? sh_atom_add_u32(&S.cnt[part[r]], 1u) : 0u;
  }
  if (!__syncthreads_or(any_sp)) return;
  if (threadIdx.x == 0 && L.level == 0 && S.first_spill) {
    S.first_spill = 0;
    atomicMin(&P.ctrl->rows_at_full, (unsigned long long)tile_row0);
  }
  const uint32_t fan = L.fan_mask + 1;
  const uint32_t dst = L.dst;
  // Partition p's thread first applies the previous spilling tile's records to
  // the chunk cursor (deferred to here so that no barrier is needed after the
  // stores), then takes this tile's count.
  for (uint32_t p = threadIdx.x; p < fan; p += THREADS) {
    const uint32_t pc = S.pend[p];
    uint32_t f = S.fill[p];
    if (pc) {
      if (f + pc > CH) {
        S.cur[p] = S.nxt[p];
        f = f + pc - CH;
      } else {
        f += pc;
      }
      S.fill[p] = f;
    }
    const uint32_t c = S.cnt[p];
    S.cnt[p] = 0;
    S.pend[p] = c;
    if (c == 0) continue;
    S.pspill[p] += c;
    if (f + c > CH) {  // this tile overflows the current chunk: open a new one
      uint32_t nc = NONE;
      const unsigned long long id = atomicAdd(&P.ctrl->pool_next[dst], 1ull);
      if (id < P.max_chunks[dst]) {
        nc = (uint32_t)id;
        P.dir_part[dst][nc] = p;
      } else {
        set_status(P.ctrl, AGG_ERR_STAGING_EXHAUSTED);
      }
      if (S.cur[p] != NONE) P.dir_count[dst][S.cur[p]] = CH;
      S.nxt[p] = nc;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    if (!sp[r]) continue;
    const uint32_t p = part[r];
    const uint32_t pos = S.fill[p] + rank[r];
    uint32_t chunk, at;
    if (pos < CH) {
      chunk = S.cur[p];
      at = pos;
    } else {
      chunk = S.nxt[p];
      at = pos - CH;
    }
    if (chunk == NONE) continue;
    longlong2 rec;
    rec.x = k[r];
    rec.y = v[r];
    __stcs(reinterpret_cast<longlong2*>(P.stg[dst] + ((size_t)chunk * CH + at) * REC_BYTES), rec);
  }
}

// Closes every open staging chunk of this block (writes its record count).
__device__ void finalize_chunks(const HashParams& P, Smem& S, uint32_t dst, uint32_t level) {
  __syncthreads();
  for (uint32_t p = threadIdx.x; p < MAX_FAN; p += THREADS) {
    uint32_t cur = S.cur[p], f = S.fill[p];
    const uint32_t pc = S.pend[p];
    if (pc) {  // the last spilling tile's records
      if (f + pc > CH) {
        cur = S.nxt[p];
        f = f + pc - CH;
      } else {
        f += pc;
      }
    }
    if (cur != NONE) P.dir_count[dst][cur] = f;
    S.cur[p] = NONE;
    S.fill[p] = CH;
    S.cnt[p] = 0;
    S.pend[p] = 0;
    if (S.pspill[p]) atomicAdd(&P.ctrl->spill_records[level], S.pspill[p]);
    S.pspill[p] = 0;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- emit

__device__ uint32_t block_exclusive_scan(uint32_t x, uint32_t& total, Smem& S) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL_MASK, inc, o);
    if ((int)lane >= o) inc += y;
  }
  if (lane == 31) S.warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < WARPS ? S.warp_tot[lane] : 0;
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL_MASK, ti, o);
      if ((int)lane >= o) ti += y;
    }
    if (lane < WARPS) S.warp_tot[lane] = ti - t;  // exclusive
    if (lane == WARPS - 1) S.scan_total = ti;
  }
  __syncthreads();
  total = S.scan_total;
  const uint32_t r = S.warp_tot[warp] + inc - x;
  __syncthreads();
  return r;
}

template <int ENT>
__device__ void emit_one(const HashParams& P, uint8_t* e, unsigned long long pos) {
  long long key, mn, mx;
  unsigned long long c, s;
  Ent<ENT>::read(e, key, c, s, mn, mx);
  if (pos < P.o_cap) {
    P.o_keys[pos] = key;
    if (P.o_count) P.o_count[pos] = c;
    if (P.o_sum) P.o_sum[pos] = (long long)s;
    if (P.o_min) P.o_min[pos] = mn;
    if (P.o_max) P.o_max[pos] = mx;
  } else {
    set_status(P.ctrl, AGG_ERR_OUTPUT_CAPACITY);
  }
  Ent<ENT>::reset(e);
}

// Clears the whole shared-memory table.
__device__ __forceinline__ void cache_reset_all(const Cache& cc, Smem& S, bool mm) {
  for (uint32_t i = threadIdx.x; i < cc.n; i += THREADS) {
    cc.key[i] = SKEY_EMPTY;
    cc.cnt[i] = 0;
    cc.sum[i] = 0;
    if (mm) {
      cc.mn[i] = INT64_MAX;
      cc.mx[i] = INT64_MIN;
    }
  }
}

// Writes every occupied slot of the active table (and the side slot) to the
// output and resets them.  The table is cut into segments of THREADS * 4 tag
// words; a block scan over each segment reserves its output rows with one
// atomic.  When the shared-memory table is idle (it is at every call) and large
// enough, the segment's occupied slots are first listed in it, and the block's
// threads then emit the list in stride, so that no thread serialises the
// entries of a dense stretch of the table; the idle table is cleared after.
template <int ENT>
__device__ void emit_table(const HashParams& P, const Team& T, const Cache& cc, uint32_t s_act, uint32_t level,
                           Smem& S) {
  const uint32_t words = s_act / 4;
  constexpr uint32_t WPT = 4;  // tag words per thread
  const uint32_t seg_words = THREADS * WPT;
  uint32_t* list = reinterpret_cast<uint32_t*>(cc.key);  // key and sum (and min, max) arrays are contiguous
  const bool use_list = (uint64_t)cc.n * (Ent<ENT>::MM ? 8u : 4u) >= (uint64_t)seg_words * 4;
  for (uint32_t seg = T.bid; (uint64_t)seg * seg_words < words; seg += T.nb) {
    const uint32_t w0 = seg * seg_words + threadIdx.x * WPT;
    uint32_t tw[WPT];
    uint32_t oc = 0;
    if (w0 + WPT <= words) {
      const uint4 t = __ldcg(reinterpret_cast<const uint4*>(P.tags + w0));
      tw[0] = t.x;
      tw[1] = t.y;
      tw[2] = t.z;
      tw[3] = t.w;
    } else {
#pragma unroll
      for (uint32_t q = 0; q < WPT; ++q) tw[q] = (w0 + q < words) ? __ldcg(P.tags + w0 + q) : 0u;
    }
#pragma unroll
    for (uint32_t q = 0; q < WPT; ++q) oc += __popc(~__vcmpeq4(tw[q], 0u) & 0x01010101u);
    uint32_t total;
    const uint32_t off = block_exclusive_scan(oc, total, S);
    if (threadIdx.x == 0) {
      S.scan_base = total ? atomicAdd(&P.ctrl->out_count, (unsigned long long)total) : 0ull;
      if (total) atomicAdd(&P.ctrl->resident_groups[level], (unsigned long long)total);
    }
    if (use_list) {
      uint32_t o = off;
#pragma unroll
      for (uint32_t q = 0; q < WPT; ++q) {
        if (tw[q] == 0) continue;
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j)
          if ((tw[q] >> (8 * j)) & 0xFFu) list[o++] = (w0 + q) * 4 + j;
        __stcg(P.tags + w0 + q, 0u);
      }
      __syncthreads();  // list and scan_base complete
      const unsigned long long base = S.scan_base;
      for (uint32_t i = threadIdx.x; i < total; i += THREADS) emit_one<ENT>(P, Ent<ENT>::at(P.ent, list[i]), base + i);
      __syncthreads();  // list free for the next segment
      continue;
    }
    __syncthreads();
    unsigned long long pos = S.scan_base + off;
#pragma unroll
    for (uint32_t q = 0; q < WPT; ++q) {
      if (tw[q] == 0) continue;
#pragma unroll
      for (uint32_t j = 0; j < 4; ++j) {
        if (((tw[q] >> (8 * j)) & 0xFFu) == 0) continue;
        emit_one<ENT>(P, Ent<ENT>::at(P.ent, (w0 + q) * 4 + j), pos);
        ++pos;
      }
      __stcg(P.tags + w0 + q, 0u);
    }
    __syncthreads();
  }
  if (use_list) {  // the shared-memory table served as the list: clear it
    cache_reset_all(cc, S, Ent<ENT>::MM);
    __syncthreads();
  }
  // the side slot of the empty-marker key
  if (T.bid == T.nb - 1 && threadIdx.x == 0) {
    uint8_t* tb = reinterpret_cast<uint8_t*>(P.tags) + P.slots;
    if (__ldcg(tb)) {
      const unsigned long long pos = atomicAdd(&P.ctrl->out_count, 1ull);
      atomicAdd(&P.ctrl->resident_groups[level], 1ull);
      emit_one<ENT>(P, Ent<ENT>::at(P.ent, P.slots), pos);
      __stcg(reinterpret_cast<long long*>(Ent<ENT>::at(P.ent, P.slots)), (long long)EMPTY_KEY);
      __stcg(tb, (uint8_t)0);
    }
  }
}


// ---------------------------------------------------------------- shared-memory rounds

// Aggregates one record into the block's shared-memory sub-partition table.
// A key may occupy only the first free slot of its 16-slot probe window, and
// slots are not freed while the sub-partition is processed, so a key that finds
// its window full of other keys never enters the table later: all of its rows
// overflow consistently (to the global table).  The window is read four slots
// (32 bytes) at a time, so that most probes finish in one step.  Returns false
// on overflow.
template <int ENT>
__device__ __forceinline__ bool sub_upsert(const Cache& cc, long long key, uint64_t h, long long v) {
  if (key == SKEY_EMPTY) return false;
  uint32_t g = ((uint32_t)(h >> 32) & (cc.n / 4 - 1)) * 4;
#pragma unroll 1
  for (int step = 0; step < 4; ++step) {
    long long kk[4];
    sh_ld_volatile_s64x2(cc.key + g, kk[0], kk[1]);
    sh_ld_volatile_s64x2(cc.key + g + 2, kk[2], kk[3]);
    int idx = -1;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      if (idx >= 0) continue;
      long long x = kk[w];
      if (x == SKEY_EMPTY) {
        x = sh_cas_s64(cc.key + g + w, SKEY_EMPTY, key);
        if (x == SKEY_EMPTY) x = key;
      }
      if (x == key) idx = (int)(g + w);
    }
    if (idx >= 0) {
      sh_red_add_u32(cc.cnt + idx, 1u);
      smem_add_u64(cc.sum + idx, (unsigned long long)v);
      if (Ent<ENT>::MM) {
        sh_min_s64(cc.mn + idx, v);
        sh_max_s64(cc.mx + idx, v);
      }
      return true;
    }
    g = (g + 4) & (cc.n - 1);
  }
  return false;
}

// As sub_upsert, for a partial state of c rows (sum s, extremes mn and mx).
template <int ENT>
__device__ __forceinline__ bool sub_upsert_part(const Cache& cc, long long key, uint64_t h, uint32_t c,
                                                unsigned long long s, long long mn, long long mx) {
  if (key == SKEY_EMPTY) return false;
  uint32_t g = ((uint32_t)(h >> 32) & (cc.n / 4 - 1)) * 4;
#pragma unroll 1
  for (int step = 0; step < 4; ++step) {
    long long kk[4];
    sh_ld_volatile_s64x2(cc.key + g, kk[0], kk[1]);
    sh_ld_volatile_s64x2(cc.key + g + 2, kk[2], kk[3]);
    int idx = -1;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      if (idx >= 0) continue;
      long long x = kk[w];
      if (x == SKEY_EMPTY) {
        x = sh_cas_s64(cc.key + g + w, SKEY_EMPTY, key);
        if (x == SKEY_EMPTY) x = key;
      }
      if (x == key) idx = (int)(g + w);
    }
    if (idx >= 0) {
      sh_red_add_u32(cc.cnt + idx, c);
      smem_add_u64(cc.sum + idx, s);
      if (Ent<ENT>::MM) {
        sh_min_s64(cc.mn + idx, mn);
        sh_max_s64(cc.mx + idx, mx);
      }
      return true;
    }
    g = (g + 4) & (cc.n - 1);
  }
  return false;
}

// Writes the groups of the shared-memory table to the output and clears it.
// Each warp takes a contiguous slice of the slots and reserves its output rows
// with one atomic of its own, so that no block-wide scan is needed; one block
// barrier at the end keeps the next sub-partition off the table until it is
// clear.  Returns the groups this thread's warp wrote (lane 0; 0 elsewhere).
template <int ENT>
__device__ uint32_t sub_emit(const HashParams& P, const Cache& cc, uint32_t level) {
  constexpr int SPL = 4;  // slots per lane in one pass of a warp (slices of 32 * SPL slots)
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t slice = cc.n / WARPS;  // multiple of 32 * SPL for n >= 2048; a loop covers the rest
  uint32_t mine = 0;
  for (uint32_t b0 = warp * slice; b0 < (warp + 1) * slice; b0 += 32 * SPL) {
    long long key[SPL];
    uint32_t occ[SPL], tot = 0;
#pragma unroll
    for (int q = 0; q < SPL; ++q) {
      const uint32_t j = b0 + q * 32 + lane;
      key[q] = j < (warp + 1) * slice ? cc.key[j] : SKEY_EMPTY;
      occ[q] = __ballot_sync(FULL_MASK, key[q] != SKEY_EMPTY);
      tot += __popc(occ[q]);
    }
    if (tot == 0) continue;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&P.ctrl->out_count, (unsigned long long)tot);
    base = __shfl_sync(FULL_MASK, base, 0);
    mine += tot;
    uint32_t before = 0;
#pragma unroll
    for (int q = 0; q < SPL; ++q) {
      const uint32_t j = b0 + q * 32 + lane;
      if (key[q] != SKEY_EMPTY) {
        const unsigned long long pos = base + before + __popc(occ[q] & lanemask_lt());
        if (pos < P.o_cap) {
          P.o_keys[pos] = key[q];
          if (P.o_count) P.o_count[pos] = cc.cnt[j];
          if (P.o_sum) P.o_sum[pos] = (long long)cc.sum[j];
          if (Ent<ENT>::MM) {
            if (P.o_min) P.o_min[pos] = cc.mn[j];
            if (P.o_max) P.o_max[pos] = cc.mx[j];
          }
        } else {
          set_status(P.ctrl, AGG_ERR_OUTPUT_CAPACITY);
        }
        cc.key[j] = SKEY_EMPTY;
        cc.cnt[j] = 0;
        cc.sum[j] = 0;
        if (Ent<ENT>::MM) {
          cc.mn[j] = INT64_MAX;
          cc.mx[j] = INT64_MIN;
        }
      }
      before += __popc(occ[q]);
    }
  }
  if (lane == 0 && mine) atomicAdd(&P.ctrl->resident_groups[level], (unsigned long long)mine);
  __syncthreads();
  return lane == 0 ? mine : 0u;
}

// Sub-partition of a record within its round (hash bits 16..31, independent of
// the bucket bits 32..63, the tag bits 0..7 and the partition bits 8..15).
__device__ __forceinline__ uint32_t sub_of(uint64_t h, uint32_t nsub) {
  return (uint32_t)((((h >> 16) & 0xFFFFull) * nsub) >> 16);
}

// Loads record r of chunk-tile t of a round (one tile is one staging chunk).
__device__ __forceinline__ bool load_chunk_record(const HashParams& P, uint32_t src, const uint32_t* list,
                                                  const uint32_t* dcount, uint32_t c0, uint64_t t, int r,
                                                  long long& k, long long& v) {
  const uint32_t chunk = __ldcg(list + c0 + (uint32_t)t);
  const uint32_t off = (uint32_t)r * THREADS + threadIdx.x;
  if (off >= __ldcg(dcount + chunk)) return false;
  const longlong2 rec = __ldcs(reinterpret_cast<const longlong2*>(P.stg[src] + ((size_t)chunk * CH + off) * REC_BYTES));
  k = rec.x;
  v = rec.y;
  return true;
}

// Stages the chunk id and record count of this block's tiles tb, tb + nb, ...
// (TLIST of them) of a round in shared memory, so that the record loads of a
// tile do not wait on two dependent loads of the chunk directory.  Returns the
// number of staged tiles.  Block-uniform call.
__device__ uint32_t stage_tiles(const Team& T, Smem& S, const uint32_t* list, const uint32_t* dcount, uint32_t c0,
                                uint64_t ntiles, uint64_t tb) {
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < TLIST; j += THREADS) {
    const uint64_t t = tb + (uint64_t)j * T.nb;
    uint32_t ch = 0, cnt = 0;
    if (t < ntiles) {
      ch = __ldcg(list + c0 + (uint32_t)t);
      cnt = __ldcg(dcount + ch);
    }
    S.tl_chunk[j] = ch;
    S.tl_count[j] = cnt;
  }
  __syncthreads();
  const uint64_t left = (ntiles - tb + T.nb - 1) / T.nb;
  return left < TLIST ? (uint32_t)left : TLIST;
}

// Record `off` of staged tile j (false past the tile's count).
__device__ __forceinline__ bool staged_record(const HashParams& P, uint32_t src, const Smem& S, uint32_t j,
                                              uint32_t off, long long& k, long long& v, bool keep_in_l2) {
  if (off >= S.tl_count[j]) return false;
  const longlong2* a = reinterpret_cast<const longlong2*>(P.stg[src] + ((size_t)S.tl_chunk[j] * CH + off) * REC_BYTES);
  const longlong2 rec = keep_in_l2 ? __ldcg(a) : __ldcs(a);
  k = rec.x;
  v = rec.y;
  return true;
}

__device__ __forceinline__ void prefetch_staged(const HashParams& P, uint32_t src, const Smem& S, uint32_t j) {
  if (P.stg_host) return;  // staging in host memory: no bulk staging in L2
  prefetch_l2(P.stg[src] + (size_t)S.tl_chunk[j] * CH * REC_BYTES, S.tl_count[j] * (uint32_t)REC_BYTES);
}

// One shared-memory round over the chunks [c0, c1) of the source area holding
// `tot` records.  Pass A: every block counts its records per sub-partition and
// stores its counts as one row of the histogram matrix `hrows` (team blocks ×
// sub-partitions, row stride `hstride` words).  Scan: the team turns the
// columns into per-block exclusive offsets in place and stores each column's
// total.  Pass B: every block scatters its records into the scratch memory
// grouped by sub-partition, through block-private cursors in shared memory
// (start of the sub-partition + this block's offset in it), so neither pass
// needs a global atomic.  Pass C lets each block aggregate whole
// sub-partitions in its shared-memory table and emit them.  Keys that overflow
// a block's table go to the level's global table G (or spill further).  Three
// grid barriers per round; pass C needs none before the next round's pass A.
template <int ENT>
__device__ bool smem_round(const HashParams& P, const Team& T, Timer& tm, const Level& G, Smem& S, const Cache& cc,
                           uint32_t src, uint32_t c0, uint32_t c1, uint64_t tot, uint32_t par, longlong2* scratch,
                           uint32_t* hrows, uint32_t hstride) {
  Ctrl* C = P.ctrl;
  const uint32_t* dcount = P.dir_count[src];
  const uint32_t* list = P.list[src];
  const uint64_t ntiles = c1 - c0;
  // sub-partitions sized by the keys-per-record of completed rounds of this parity
  const double recd = (double)ld_relaxed_u64(&C->lvl_sub_records[par]);
  const double grpd = (double)ld_relaxed_u64(&C->lvl_sub_groups[par]);
  double est = recd > 0 ? 1.3 * grpd / recd + 0.02 : 1.0;
  if (est > 1.0) est = 1.0;
  const double subkeys = 0.55 * (double)cc.n;
  uint64_t nsub = (uint64_t)((double)tot * est / subkeys) + 1;
  const uint64_t nsub_cap = (2ull * cc.n < hstride) ? 2ull * cc.n : hstride;
  if (nsub > nsub_cap) nsub = nsub_cap;
  uint32_t* hist = reinterpret_cast<uint32_t*>(cc.key);  // pass A: counts; pass B: sub-partition starts
  uint32_t* cur = reinterpret_cast<uint32_t*>(cc.sum);   // pass B: this block's write cursors
  uint32_t* myrow = hrows + (size_t)T.bid * hstride;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // ---- pass A: records per sub-partition, one histogram row per block
  for (uint32_t i = threadIdx.x; i < nsub; i += THREADS) hist[i] = 0;
  for (uint64_t tb = T.bid; tb < ntiles; tb += (uint64_t)TLIST * T.nb) {
    const uint32_t nj = stage_tiles(T, S, list, dcount, c0, ntiles, tb);
    if (threadIdx.x < A_TILES && threadIdx.x < nj) prefetch_staged(P, src, S, threadIdx.x);
    for (uint32_t j = 0; j < nj; j += A_TILES) {  // A_TILES tiles per step: A_TILES * RPT loads in flight
      if (threadIdx.x < A_TILES && j + A_TILES + threadIdx.x < nj) prefetch_staged(P, src, S, j + A_TILES + threadIdx.x);
      long long k[A_TILES * RPT];
      bool ok[A_TILES * RPT];
#pragma unroll
      for (int r = 0; r < A_TILES * RPT; ++r) {  // keys only
        const uint32_t jj = j + (uint32_t)(r / RPT);
        const uint32_t off = (uint32_t)(r % RPT) * THREADS + threadIdx.x;
        ok[r] = jj < nj && off < S.tl_count[jj];
        k[r] = ok[r] ? __ldcs(reinterpret_cast<const long long*>(P.stg[src] +
                                                                 ((size_t)S.tl_chunk[jj] * CH + off) * REC_BYTES))
                     : 0;
      }
#pragma unroll
      for (int r = 0; r < A_TILES * RPT; ++r)
        if (ok[r]) sh_red_add_u32(&hist[sub_of(fmix64((uint64_t)k[r] ^ G.seed), (uint32_t)nsub)], 1u);
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nsub; i += THREADS) __stcg(myrow + i, hist[i]);
  if (!grid_barrier(T, C, P.timeout_ns, S)) return false;

  // this round's pass-C claim counter (its parity was last used two rounds ago)
  if (T.bid == 0 && threadIdx.x == 0) C->sub_next[par] = 0;
  // ---- scan: a block takes 32 columns at a time; its warps split the team's
  // rows, sum their share, exchange the sums, then write the exclusive offsets
  {
    uint32_t* wsum = reinterpret_cast<uint32_t*>(cc.key);  // WARPS x 32 partial sums
    const uint32_t rpw = (T.nb + WARPS - 1) / WARPS;
    const uint32_t b0 = warp * rpw, b1 = b0 + rpw < T.nb ? b0 + rpw : T.nb;
    for (uint64_t g = T.bid; g * 32 < nsub; g += T.nb) {
      const uint32_t col = (uint32_t)g * 32 + lane;
      uint32_t part = 0;
      if (col < nsub)
        for (uint32_t b = b0; b < b1; ++b) part += __ldcg(hrows + (size_t)b * hstride + col);
      wsum[warp * 32 + lane] = part;
      __syncthreads();
      uint32_t acc = 0;
      for (uint32_t w = 0; w < warp; ++w) acc += wsum[w * 32 + lane];
      if (col < nsub) {
        if (warp == WARPS - 1) __stcg(&C->sub_tot[par][col], acc + part);
        for (uint32_t b = b0; b < b1; ++b) {
          uint32_t* q = hrows + (size_t)b * hstride + col;
          const uint32_t x = __ldcg(q);
          __stcg(q, acc);
          acc += x;
        }
      }
      __syncthreads();
    }
  }
  if (!grid_barrier(T, C, P.timeout_ns, S)) return false;
  tm.lap(T, C, PH_SUB_COUNT);

  // ---- pass B: sub-partition starts, this block's cursors, then the scatter
  {
    const uint32_t per = (uint32_t)((nsub + THREADS - 1) / THREADS);
    const uint32_t s0 = threadIdx.x * per;
    uint32_t mine = 0;
    for (uint32_t i = 0; i < per; ++i)
      if (s0 + i < nsub) mine += __ldcg(&C->sub_tot[par][s0 + i]);
    uint32_t total;
    uint32_t acc = block_exclusive_scan(mine, total, S);
    for (uint32_t i = 0; i < per; ++i) {
      if (s0 + i >= nsub) break;
      hist[s0 + i] = acc;
      if (T.bid == 0) C->sub_base[par][s0 + i] = acc;
      acc += __ldcg(&C->sub_tot[par][s0 + i]);
    }
    if (T.bid == 0 && threadIdx.x == 0) C->sub_base[par][nsub] = total;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nsub; i += THREADS) cur[i] = hist[i] + __ldcg(myrow + i);
    __syncthreads();
  }
  for (uint64_t tb = T.bid; tb < ntiles; tb += (uint64_t)TLIST * T.nb) {
   const uint32_t nj = stage_tiles(T, S, list, dcount, c0, ntiles, tb);
   for (uint32_t j = 0; j < nj; ++j) {
    if (threadIdx.x == 0 && j + 1 < nj) prefetch_staged(P, src, S, j + 1);
    long long k[RPT], v[RPT];
    uint32_t sb[RPT];
    bool ok[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
      ok[r] = staged_record(P, src, S, j, (uint32_t)r * THREADS + threadIdx.x, k[r], v[r], false);
#pragma unroll
    for (int r = 0; r < RPT; ++r) sb[r] = ok[r] ? sub_of(fmix64((uint64_t)k[r] ^ G.seed), (uint32_t)nsub) : 0u;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      // one shared-memory atomic per record: lanes rarely share one of the
      // round's ~thousand sub-partitions, and __match_any_sync costs more
      if (ok[r]) {
        const uint64_t at = sh_atom_add_u32(&cur[sb[r]], 1u);
        longlong2 rec;
        rec.x = k[r];
        rec.y = v[r];
        if (at < tot) scratch[at] = rec;
        else set_status(C, AGG_ERR_INTERNAL);
      }
    }
   }
  }
  if (!grid_barrier(T, C, P.timeout_ns, S)) return false;
  tm.lap(T, C, PH_SUB_SCATTER);

  // ---- pass C: whole sub-partitions aggregated in shared memory
  // Sub-partitions are claimed dynamically (one ahead), so that blocks that
  // drew small ones take more.
  cache_reset_all(cc, S, Ent<ENT>::MM);
  if (threadIdx.x == 0) S.sub_q[0] = atomicAdd(&C->sub_next[par], 1u);
  unsigned long long my_recs = 0, my_groups = 0;
  __syncthreads();
  // each iteration ends with sub_emit's barrier, which also publishes the
  // sub-partition claimed for the next iteration
  for (uint32_t it = 0;; ++it) {
    const uint32_t sbi = S.sub_q[it & 1];
    if (sbi >= nsub) break;
    if (threadIdx.x == 0) {
      // claim the next sub-partition and stage its records in L2 while this one runs
      const uint32_t nx = atomicAdd(&C->sub_next[par], 1u);
      S.sub_q[(it + 1) & 1] = nx;
      if (AGG_PASSC_PREFETCH && nx < nsub) {
        const uint32_t a = __ldcg(&C->sub_base[par][nx]), b = __ldcg(&C->sub_base[par][nx + 1]);
        if (a < b && b <= tot) {
          for (uint32_t o = a; o < b; o += 4096)  // bulk prefetches of at most 64 KiB
            prefetch_l2(scratch + o, (b - o < 4096u ? b - o : 4096u) * (uint32_t)REC_BYTES);
        }
      }
    }
    uint32_t lo = __ldcg(&C->sub_base[par][sbi]), hi = __ldcg(&C->sub_base[par][sbi + 1]);
    if (hi > tot || lo > hi) {  // inconsistent offsets: report, never read past the scratch
      if (threadIdx.x == 0) set_status(C, AGG_ERR_INTERNAL);
      lo = hi = 0;
    }
    bool overflow = false;
    for (uint32_t t0 = lo; t0 < hi; t0 += TILE) {
      long long k[RPT], v[RPT];
      uint64_t h[RPT];
      bool need[RPT], in[RPT];
#pragma unroll
      for (int r = 0; r < RPT; ++r) {  // all loads first
        const uint32_t i = t0 + (uint32_t)r * THREADS + threadIdx.x;
        in[r] = i < hi;
        k[r] = 0;
        v[r] = 0;
        if (in[r]) {
          const longlong2 rec = scratch[i];
          k[r] = rec.x;
          v[r] = rec.y;
        }
      }
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        h[r] = fmix64((uint64_t)k[r] ^ G.seed);
        need[r] = in[r] && !sub_upsert<ENT>(cc, k[r], h[r], v[r]);
        overflow |= need[r];
      }
      global_and_spill<ENT>(P, G, S, cc, k, v, h, need, in, 0, false);
    }
    if (overflow) atomicOr(&C->overflow_used[G.level & 1], 1u);
    if (lo == hi) __syncthreads();  // else the last tile's vote in global_and_spill ordered every upsert before the emit
    my_groups += sub_emit<ENT>(P, cc, G.level);
    my_recs += hi - lo;
  }
  if (threadIdx.x == 0 && my_recs) atomicAdd(&C->lvl_sub_records[par], my_recs);
  if (my_groups) atomicAdd(&C->lvl_sub_groups[par], my_groups);  // lane 0 of each warp
  cache_reset_all(cc, S, Ent<ENT>::MM);
  __syncthreads();
  tm.lap(T, C, PH_SUB_AGG);
  return true;
}

// Restores the entries that served as scratch to the empty state.
template <int ENT>
__device__ void restore_scratch(const HashParams& P, const Team& T, uint32_t gslots) {
  for (uint64_t s = gslots + T.bid * (uint64_t)THREADS + threadIdx.x; s < P.slots;
       s += (uint64_t)T.nb * THREADS)
    Ent<ENT>::reset(Ent<ENT>::at(P.ent, (uint32_t)s));
}

// Last block to arrive publishes the group count and the run's statistics,
// then zeroes the per-run control fields for the next run.
__device__ void final_step(const HashParams& P, const Team& T, uint32_t levels) {
  __syncthreads();
  if (threadIdx.x != 0) return;
  Ctrl* C = P.ctrl;
  __threadfence();
  const uint32_t prev = atomicAdd(&C->done_count, 1u);
  if (prev != T.nb - 1) return;
  __threadfence();
  volatile Ctrl* V = C;
  const unsigned long long ng = V->out_count;
  if (P.o_ngroups) *P.o_ngroups = ng;
  C->last_n_rows = P.n;
  C->last_n_groups = ng;
  C->last_levels = levels;
  C->last_rounds = V->rounds;
  C->last_rows_at_full = V->rows_at_full;
  for (int l = 0; l < AGG_MAX_LEVELS; ++l) {
    C->last_spill_records[l] = V->spill_records[l];
    C->last_resident_groups[l] = V->resident_groups[l];
    C->spill_records[l] = 0;
    C->resident_groups[l] = 0;
  }
  for (int ph = 0; ph < PHASES; ++ph) {
    C->last_phase_ns[ph] = V->phase_ns[ph];
    C->phase_ns[ph] = 0;
  }
  C->last_sorted = V->sorted_used;
  C->sorted_used = 0;
  C->sorted_fail = 0;
  C->last_fallback_records = V->fallback_records;
  C->last_fallback_level = V->fallback_level;
  C->fallback_records = 0;
  C->fallback_level = 0;
  C->fallback_now = 0;
  C->occupancy = 0;
  C->out_count = 0;
  C->pool_next[0] = 0;
  C->pool_next[1] = 0;
  C->rows_at_full = ~0ull;
  C->tile_next = 0;
  C->rounds = 0;
  for (int s = 0; s < 2; ++s)
    for (int p = 0; p < MAX_FAN; ++p) {
      C->part_records[s][p] = 0;
      C->part_chunks[s][p] = 0;
      C->part_cursor[s][p] = 0;
    }
  __threadfence();
  C->done_count = 0;
}


// ---------------------------------------------------------------- sorted-input path

// Sort-based aggregation needs no table when its input is already sorted
// (Section 6.4: on sorted data the Sort-based algorithm wins, its sort phase
// degenerating to a scan).  The persistent kernel therefore first checks a
// sample: every block reads the same THREADS evenly spaced adjacent key pairs
// and the order of the pairs' first keys, so all blocks reach the same verdict
// with no barrier.  If the sample is in order the run tries the sorted path,
// on contiguous row ranges, one per block:
//   S1  each block checks its rows are non-decreasing and counts the segment
//       heads (a row whose key differs from its predecessor's); a descent
//       anywhere sets a flag, and after a grid barrier every block falls back
//       to the hash path;
//   S2  each block's first output row is the number of heads before its range;
//   S3  a block-wide segmented scan of (COUNT, SUM, MIN, MAX), carried from
//       tile to tile, gives each segment's aggregate at its last row, which is
//       stored at the segment's head rank when the head lies in the block; a
//       segment that starts in an earlier block leaves its partial aggregate
//       (the block's leading partial) aside;
//   S4  after a grid barrier, each leading partial is added to its segment's
//       row with atomics (COUNT and SUM added, MIN and MAX combined).
// The output is in ascending key order.

struct Seg {
  unsigned long long c, s;
  long long mn, mx;
  uint32_t f;  // the span holds a segment head
};

__device__ __forceinline__ Seg seg_identity() { return Seg{0ull, 0ull, INT64_MAX, INT64_MIN, 0u}; }

// a followed by b
__device__ __forceinline__ Seg seg_combine(const Seg& a, const Seg& b) {
  if (b.f) return b;
  return Seg{a.c + b.c, a.s + b.s, a.mn < b.mn ? a.mn : b.mn, a.mx > b.mx ? a.mx : b.mx, a.f};
}

__device__ __forceinline__ Seg seg_shfl_up(const Seg& x, int o) {
  return Seg{__shfl_up_sync(FULL_MASK, x.c, o), __shfl_up_sync(FULL_MASK, x.s, o), __shfl_up_sync(FULL_MASK, x.mn, o),
             __shfl_up_sync(FULL_MASK, x.mx, o), __shfl_up_sync(FULL_MASK, x.f, o)};
}

// The same sample in every block: true when it shows no descent.
__device__ __noinline__ bool sorted_sample(const HashParams& P, Smem& S) {
  const uint64_t n = P.n;
  const uint64_t j = (n - 2) * threadIdx.x / (THREADS - 1);  // 0 .. n-2
  const long long a = __ldcg(P.keys + j), b = __ldcg(P.keys + j + 1);
  bool ok = a <= b;
  const long long nb = __shfl_down_sync(FULL_MASK, a, 1);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < 31) ok = ok && a <= nb;
  if (lane == 0) S.sw_mn[warp] = a;
  __syncthreads();
  if (lane == 31 && warp + 1 < WARPS) ok = ok && a <= S.sw_mn[warp + 1];
  return __syncthreads_and(ok) != 0;
}

// Row sources of the segmented reduction: the caller's input (keys and
// values of type VT), or records (key, int64 value) of a contiguous buffer.
template <int VT>
struct InputRows {
  const HashParams& P;
  __device__ long long key(uint64_t i) const { return __ldcg(P.keys + i); }
  __device__ __forceinline__ void load4(uint64_t row, uint64_t r1, long long (&k)[4], long long (&v)[4],
                                        bool with_vals) const {
    if (P.vec_ok && row + 3 < r1) {
      const longlong2 k01 = __ldcs(reinterpret_cast<const longlong2*>(P.keys + row));
      const longlong2 k23 = __ldcs(reinterpret_cast<const longlong2*>(P.keys + row + 2));
      k[0] = k01.x;
      k[1] = k01.y;
      k[2] = k23.x;
      k[3] = k23.y;
      if (!with_vals || !P.has_vals) {
        v[0] = v[1] = v[2] = v[3] = 0;
      } else if (VT == AGG_I64) {
        const longlong2 v01 = __ldcs(reinterpret_cast<const longlong2*>(static_cast<const long long*>(P.vals) + row));
        const longlong2 v23 =
            __ldcs(reinterpret_cast<const longlong2*>(static_cast<const long long*>(P.vals) + row + 2));
        v[0] = v01.x;
        v[1] = v01.y;
        v[2] = v23.x;
        v[3] = v23.y;
      } else {
        const int2 v01 = __ldcs(reinterpret_cast<const int2*>(static_cast<const int*>(P.vals) + row));
        const int2 v23 = __ldcs(reinterpret_cast<const int2*>(static_cast<const int*>(P.vals) + row + 2));
        v[0] = v01.x;
        v[1] = v01.y;
        v[2] = v23.x;
        v[3] = v23.y;
      }
      return;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      k[j] = 0;
      v[j] = 0;
      if (row + j < r1) {
        k[j] = __ldcs(P.keys + row + j);
        if (with_vals && P.has_vals)
          v[j] = VT == AGG_I64 ? __ldcs(static_cast<const long long*>(P.vals) + row + j)
                               : (long long)__ldcs(static_cast<const int*>(P.vals) + row + j);
      }
    }
  }
  __device__ void prefetch(uint64_t row, uint64_t rows, bool with_vals) const {
    prefetch_l2(P.keys + row, (uint32_t)(rows * 8));
    if (with_vals && P.has_vals)
      prefetch_l2(static_cast<const char*>(P.vals) + row * (VT == AGG_I64 ? 8 : 4), (uint32_t)(rows * (VT == AGG_I64 ? 8 : 4)));
  }
};

struct RecordRows {
  const longlong2* rec;
  __device__ long long key(uint64_t i) const { return __ldcg(&rec[i].x); }
  __device__ __forceinline__ void load4(uint64_t row, uint64_t r1, long long (&k)[4], long long (&v)[4], bool) const {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      k[j] = 0;
      v[j] = 0;
      if (row + j < r1) {
        const longlong2 x = __ldcs(rec + row + j);
        k[j] = x.x;
        v[j] = x.y;
      }
    }
  }
  __device__ void prefetch(uint64_t row, uint64_t rows, bool) const { prefetch_l2(rec + row, (uint32_t)(rows * 16)); }
};

// Segmented reduction of n rows in non-decreasing key order (checked when
// check_order is set: a descent makes it return 0 after a grid barrier, with
// nothing written).  Groups go to the output rows out_base + head rank.
// Returns 1 when done (every block gets the group count in *groups), -1 when
// a bounded wait gave up.
template <class Rows>
__device__ __noinline__ int seg_reduce(const HashParams& P, const Team& T, Smem& S, const Rows& src, uint64_t n,
                                       bool check_order, unsigned long long out_base, unsigned long long* groups) {
  Ctrl* C = P.ctrl;
  const uint64_t per = (((n + T.nb - 1) / T.nb) + 3) & ~3ull;  // rows per block, a multiple of 4
  const uint64_t r0 = (uint64_t)T.bid * per < n ? (uint64_t)T.bid * per : n;
  const uint64_t r1 = r0 + per < n ? r0 + per : n;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // ---- S1: segment heads of this block's rows (and the order check)
  uint32_t heads = 0;
  bool bad = false;
  for (uint64_t t0 = r0; t0 < r1; t0 += TILE) {
    if (threadIdx.x == 0 && t0 + TILE < r1)
      src.prefetch(t0 + TILE, r1 - t0 - TILE < (uint64_t)TILE ? r1 - t0 - TILE : TILE, false);
    const uint64_t row = t0 + 4ull * threadIdx.x;
    long long k[4] = {0, 0, 0, 0}, v[4];
    if (row < r1) src.load4(row, r1, k, v, false);
    // the key before this thread's rows: the previous lane's last key, or a load
    const long long up = __shfl_up_sync(FULL_MASK, k[3], 1);
    if (row >= r1) continue;
    long long prev = lane > 0 ? up : (row > 0 ? src.key(row - 1) : 0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (row + j >= r1) break;
      if (row + j == 0 || k[j] != prev) ++heads;
      if (row + j > 0 && k[j] < prev) bad = true;
      prev = k[j];
    }
  }
  uint32_t total;
  block_exclusive_scan(heads, total, S);
  bad = __syncthreads_or(check_order && bad);
  if (threadIdx.x == 0) {
    C->sorted_heads[T.bid] = total;
    if (bad) atomicOr(&C->sorted_fail, 1u);
  }
  if (!grid_barrier(T, C, P.timeout_ns, S)) return -1;
  if (check_order && ld_acquire_u32(&C->sorted_fail)) return 0;

  // ---- S2: rows of the output before this block's range
  unsigned long long before = 0, all = 0;
  for (uint32_t b = threadIdx.x; b < T.nb; b += THREADS) {
    const unsigned long long h = __ldcg(&C->sorted_heads[b]);
    all += h;
    if (b < T.bid) before += h;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    before += __shfl_down_sync(FULL_MASK, before, o);
    all += __shfl_down_sync(FULL_MASK, all, o);
  }
  if (lane == 0) {
    S.sw_c[warp] = before;
    S.sw_s[warp] = all;
  }
  if (threadIdx.x == 0) {
    S.tc_c = S.tc_s = 0;
    S.tc_mn = INT64_MAX;
    S.tc_mx = INT64_MIN;
    S.tc_f = 0;
    S.lead_valid = 0;
    S.tile_prev_key = r0 > 0 && r0 < r1 ? src.key(r0 - 1) : 0;
  }
  __syncthreads();
  unsigned long long base = 0, n_groups = 0;
  for (int w = 0; w < WARPS; ++w) {
    base += S.sw_c[w];
    n_groups += S.sw_s[w];
  }
  __syncthreads();

  // ---- S3: segmented reduction, tile by tile
  unsigned long long tile_heads = 0;  // heads of this block before the current tile
  for (uint64_t t0 = r0; t0 < r1; t0 += TILE) {
    if (threadIdx.x == 0 && t0 + TILE < r1)
      src.prefetch(t0 + TILE, r1 - t0 - TILE < (uint64_t)TILE ? r1 - t0 - TILE : TILE, true);
    const uint64_t row = t0 + 4ull * threadIdx.x;
    long long k[4] = {0, 0, 0, 0}, v[4] = {0, 0, 0, 0};
    if (row < r1) src.load4(row, r1, k, v, true);
    // neighbouring keys: shuffles inside a warp, shared memory across warps,
    // one load past the tile
    const long long up = __shfl_up_sync(FULL_MASK, k[3], 1);
    const long long dn = __shfl_down_sync(FULL_MASK, k[0], 1);
    if (lane == 31) S.wl_key[warp] = k[3];
    if (lane == 0) S.wf_key[warp] = k[0];
    long long edge_next = 0;
    if (threadIdx.x == THREADS - 1 && row + 4 < n && row + 4 < r1) edge_next = src.key(row + 4);
    __syncthreads();
    const long long prev = lane > 0 ? up : (warp > 0 ? S.wl_key[warp - 1] : S.tile_prev_key);
    const long long next = lane < 31 ? dn : (warp < WARPS - 1 ? S.wf_key[warp + 1] : edge_next);
    bool valid[4], head[4], last[4];
    uint32_t my_heads = 0;
    Seg x = seg_identity();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      valid[j] = row + j < r1;
      head[j] = valid[j] && (row + j == 0 || k[j] != (j == 0 ? prev : k[j - 1]));
      const bool at_end = row + j + 1 >= r1;
      last[j] = valid[j] && (at_end || (j < 3 ? k[j + 1] != k[j] : next != k[j]));
      my_heads += head[j];
      if (valid[j]) x = seg_combine(x, Seg{1ull, (unsigned long long)v[j], v[j], v[j], head[j] ? 1u : 0u});
    }
    // warp scans of the spans and of the head counts
    Seg xi = x;
    uint32_t hi = my_heads;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const Seg y = seg_shfl_up(xi, o);
      const uint32_t hy = __shfl_up_sync(FULL_MASK, hi, o);
      if ((int)lane >= o) {
        xi = seg_combine(y, xi);
        hi += hy;
      }
    }
    Seg ex = seg_shfl_up(xi, 1);
    if (lane == 0) ex = seg_identity();
    if (lane == 31) {
      S.sw_c[warp] = xi.c;
      S.sw_s[warp] = xi.s;
      S.sw_mn[warp] = xi.mn;
      S.sw_mx[warp] = xi.mx;
      S.sw_f[warp] = xi.f;
      S.wh[warp] = hi;
    }
    __syncthreads();
    if (warp == 0) {  // carry into each warp, and into the next tile
      Seg t = lane < WARPS ? Seg{S.sw_c[lane], S.sw_s[lane], S.sw_mn[lane], S.sw_mx[lane], S.sw_f[lane]}
                           : seg_identity();
      uint32_t th = lane < WARPS ? S.wh[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const Seg y = seg_shfl_up(t, o);
        const uint32_t hy = __shfl_up_sync(FULL_MASK, th, o);
        if ((int)lane >= o) {
          t = seg_combine(y, t);
          th += hy;
        }
      }
      const Seg carry{S.tc_c, S.tc_s, S.tc_mn, S.tc_mx, S.tc_f};
      Seg wex = seg_shfl_up(t, 1);
      const uint32_t hex = __shfl_up_sync(FULL_MASK, th, 1);
      if (lane == 0) wex = seg_identity();
      const Seg cin = seg_combine(carry, wex);
      __syncwarp();
      if (lane < WARPS) {
        S.wc_c[lane] = cin.c;
        S.wc_s[lane] = cin.s;
        S.wc_mn[lane] = cin.mn;
        S.wc_mx[lane] = cin.mx;
        S.wc_f[lane] = cin.f;
        S.wh[lane] = lane == 0 ? 0u : hex;
      }
      if (lane == WARPS - 1) {
        const Seg nt = seg_combine(carry, t);
        S.tc_c = nt.c;
        S.tc_s = nt.s;
        S.tc_mn = nt.mn;
        S.tc_mx = nt.mx;
        S.tc_f = nt.f;
        S.wh[WARPS] = th;
      }
    }
    __syncthreads();
    Seg acc = seg_combine(Seg{S.wc_c[warp], S.wc_s[warp], S.wc_mn[warp], S.wc_mx[warp], S.wc_f[warp]}, ex);
    unsigned long long hidx = base + tile_heads + S.wh[warp] + (hi - my_heads);  // heads before this thread's rows
    const uint32_t tile_total = S.wh[WARPS];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!valid[j]) break;
      acc = seg_combine(acc, Seg{1ull, (unsigned long long)v[j], v[j], v[j], head[j] ? 1u : 0u});
      hidx += head[j];
      if (!last[j]) continue;
      if (acc.f) {  // the segment's head lies in this block: its row is complete here
        const unsigned long long pos = out_base + hidx - 1;
        if (pos < P.o_cap) {
          P.o_keys[pos] = k[j];
          if (P.o_count) P.o_count[pos] = acc.c;
          if (P.o_sum) P.o_sum[pos] = (long long)acc.s;
          if (P.o_min) P.o_min[pos] = acc.mn;
          if (P.o_max) P.o_max[pos] = acc.mx;
        } else {
          set_status(C, AGG_ERR_OUTPUT_CAPACITY);
        }
      } else {  // continues a segment of an earlier block
        S.lead_c = acc.c;
        S.lead_s = acc.s;
        S.lead_mn = acc.mn;
        S.lead_mx = acc.mx;
        S.lead_valid = 1;
      }
    }
    if (threadIdx.x == THREADS - 1) S.tile_prev_key = k[3];  // the key before the next tile
    tile_heads += tile_total;
    __syncthreads();
  }

  // ---- S4: leading partials into the rows of segments that began earlier
  if (!grid_barrier(T, C, P.timeout_ns, S)) return -1;
  if (threadIdx.x == 0 && S.lead_valid && base > 0) {
    const unsigned long long pos = out_base + base - 1;
    if (pos < P.o_cap) {
      if (P.o_count) atomicAdd(reinterpret_cast<unsigned long long*>(P.o_count + pos), S.lead_c);
      if (P.o_sum) atomicAdd(reinterpret_cast<unsigned long long*>(P.o_sum + pos), S.lead_s);
      if (P.o_min) atomicMin(reinterpret_cast<long long*>(P.o_min + pos), S.lead_mn);
      if (P.o_max) atomicMax(reinterpret_cast<long long*>(P.o_max + pos), S.lead_mx);
    }
  }
  *groups = n_groups;
  return 1;
}

// The sorted-input path over the caller's rows: 1 done, 0 not sorted (the
// hash path must run), -1 a bounded wait gave up.
template <int ENT, int VT>
__device__ int sorted_groupby(const HashParams& P, const Team& T, Smem& S) {
  unsigned long long ng = 0;
  const int r = seg_reduce(P, T, S, InputRows<VT>{P}, P.n, true, 0ull, &ng);
  if (r > 0 && T.bid == 0 && threadIdx.x == 0) {
    P.ctrl->out_count = ng;
    P.ctrl->resident_groups[0] = ng;
    P.ctrl->sorted_used = 1;
  }
  return r;
}

// ---------------------------------------------------------------- recursion fallback (sort path)

// The hybrid hash falls back to a sort-based aggregation for records that
// partitioning no longer shrinks (Section 4.3: when the grace levels exceed
// those a sort-based algorithm would need, or a partition's output is more
// than 80% of its input).  Here a level falls back when it reaches the depth
// cap, or when the records completed at the level before formed more than 0.8
// groups per record.  All of the level's records are then sorted by key with
// an LSD radix sort inside the kernel (eight passes of eight bits: a digit
// histogram per block, column scans, and a stable scatter that ranks each
// round of THREADS records by warp (__match_any_sync) and across warps), and
// reduced by segments like sorted input.  Pass 0 reads the staging chunks; the
// passes alternate between the two staging areas' data regions.

constexpr int RADIX = 256;

__device__ __forceinline__ uint32_t radix_digit(long long key, int pass) {
  return (uint32_t)((((uint64_t)key) ^ 0x8000000000000000ull) >> (8 * pass)) & 0xFFu;
}

// Stable scatter of one round: `valid` lanes hold records in input order
// (thread order); wcnt (WARPS x RADIX, zero on entry and exit), off (the
// block's next free position per digit) and rtot are in shared memory.
__device__ __forceinline__ void radix_round(bool valid, const longlong2& rec, int pass, longlong2* out, uint16_t* wcnt,
                                            uint32_t* off, uint32_t* rtot) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t d = valid ? radix_digit(rec.x, pass) : (uint32_t)RADIX + lane;  // idle lanes match no one
  const uint32_t peers = __match_any_sync(FULL_MASK, d);
  const uint32_t rank = __popc(peers & lanemask_lt());
  if (valid && rank == 0) wcnt[warp * RADIX + d] = (uint16_t)__popc(peers);
  __syncthreads();
  for (uint32_t dd = threadIdx.x; dd < (uint32_t)RADIX; dd += THREADS) {  // exclusive prefix over the warps
    uint32_t run = 0;
    for (int w = 0; w < WARPS; ++w) {
      const uint32_t c = wcnt[w * RADIX + dd];
      wcnt[w * RADIX + dd] = (uint16_t)run;
      run += c;
    }
    rtot[dd] = run;
  }
  __syncthreads();
  if (valid) out[(uint64_t)off[d] + wcnt[warp * RADIX + d] + rank] = rec;
  __syncthreads();
  for (uint32_t dd = threadIdx.x; dd < (uint32_t)RADIX; dd += THREADS) {
    off[dd] += rtot[dd];
    for (int w = 0; w < WARPS; ++w) wcnt[w * RADIX + dd] = 0;
  }
  __syncthreads();
}

// Sorts the R records of the chunks [0, nch) of staging area `src` by key
// into bufB (bufA is the other buffer).  H (team blocks x RADIX) and TOT
// (RADIX) are scratch words.  False when a bounded wait gave up.
__device__ __noinline__ bool fallback_sort(const HashParams& P, const Team& T, Smem& S, const Cache& cc, uint32_t src,
                                           uint64_t nch, uint64_t R, longlong2* bufA, longlong2* bufB, uint32_t* H,
                                           uint32_t* TOT) {
  uint16_t* wcnt = reinterpret_cast<uint16_t*>(cc.key);
  uint32_t* off = reinterpret_cast<uint32_t*>(wcnt + WARPS * RADIX);
  uint32_t* rtot = off + RADIX;
  const uint32_t* dcount = P.dir_count[src];
  const longlong2* chunks = reinterpret_cast<const longlong2*>(P.stg[src]);
  const uint64_t c0 = nch * T.bid / T.nb, c1 = nch * (T.bid + 1) / T.nb;
  const uint64_t a0 = R * T.bid / T.nb, a1 = R * (T.bid + 1) / T.nb;
  for (int pass = 0; pass < 8; ++pass) {
    const longlong2* in = (pass & 1) ? bufA : bufB;  // pass 0 reads the chunks
    longlong2* out = (pass & 1) ? bufB : bufA;
    // digit histogram of this block's records
    for (uint32_t i = threadIdx.x; i < (uint32_t)RADIX; i += THREADS) off[i] = 0;
    __syncthreads();
    if (pass == 0) {
      for (uint64_t c = c0; c < c1; ++c) {
        const uint32_t cnt = __ldcg(dcount + c);
        for (uint32_t j = threadIdx.x; j < cnt; j += THREADS)
          sh_red_add_u32(&off[radix_digit(__ldcg(&chunks[c * CH + j].x), 0)], 1u);
      }
    } else {
      for (uint64_t i = a0 + threadIdx.x; i < a1; i += THREADS) sh_red_add_u32(&off[radix_digit(__ldcg(&in[i].x), pass)], 1u);
    }
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < (uint32_t)RADIX; d += THREADS) __stcg(H + (size_t)T.bid * RADIX + d, off[d]);
    if (!grid_barrier(T, P.ctrl, P.timeout_ns, S)) return false;
    // column scans: for each digit, exclusive offsets of the blocks in order
    for (uint32_t d = T.bid; d < (uint32_t)RADIX; d += T.nb) {
      const uint32_t per = (T.nb + THREADS - 1) / THREADS, b0 = threadIdx.x * per;
      uint32_t mine = 0;
      for (uint32_t i = 0; i < per; ++i)
        if (b0 + i < T.nb) mine += __ldcg(H + (size_t)(b0 + i) * RADIX + d);
      uint32_t total;
      uint32_t ex = block_exclusive_scan(mine, total, S);
      for (uint32_t i = 0; i < per; ++i) {
        if (b0 + i >= T.nb) break;
        uint32_t* q = H + (size_t)(b0 + i) * RADIX + d;
        const uint32_t x = __ldcg(q);
        __stcg(q, ex);
        ex += x;
      }
      if (threadIdx.x == 0) __stcg(TOT + d, total);
    }
    if (!grid_barrier(T, P.ctrl, P.timeout_ns, S)) return false;
    // this block's first position for every digit
    uint32_t tt;
    const uint32_t ex = block_exclusive_scan(threadIdx.x < (uint32_t)RADIX ? __ldcg(TOT + threadIdx.x) : 0u, tt, S);
    if (threadIdx.x < (uint32_t)RADIX) off[threadIdx.x] = ex + __ldcg(H + (size_t)T.bid * RADIX + threadIdx.x);
    for (uint32_t i = threadIdx.x; i < (uint32_t)(WARPS * RADIX); i += THREADS) wcnt[i] = 0;
    __syncthreads();
    if (pass == 0) {
      for (uint64_t c = c0; c < c1; ++c) {
        const uint32_t cnt = __ldcg(dcount + c);
        for (uint32_t j0 = 0; j0 < cnt; j0 += THREADS) {
          const bool valid = j0 + threadIdx.x < cnt;
          const longlong2 rec = valid ? __ldcg(&chunks[c * CH + j0 + threadIdx.x]) : make_longlong2(0, 0);
          radix_round(valid, rec, 0, out, wcnt, off, rtot);
        }
      }
    } else {
      for (uint64_t i0 = a0; i0 < a1; i0 += THREADS) {
        const bool valid = i0 + threadIdx.x < a1;
        const longlong2 rec = valid ? __ldcg(&in[i0 + threadIdx.x]) : make_longlong2(0, 0);
        radix_round(valid, rec, pass, out, wcnt, off, rtot);
      }
    }
    if (!grid_barrier(T, P.ctrl, P.timeout_ns, S)) return false;
  }
  return true;
}

// ---------------------------------------------------------------- the kernel

// The whole group-by of one input by one team: level 0 over the input, then
// the spilled levels.  Returns false when a bounded wait gave up (the team
// must stop).
constexpr int RUN_ABORT = 0, RUN_DONE = 1, RUN_FALLBACK = 2;

template <int ENT, int VT>
__device__ int run_groupby(const HashParams& P, const Team& T, Smem& S, const Cache& cc) {
  Ctrl* C = P.ctrl;
  const uint32_t fan = 1u << P.fan_log2;
  Timer tm, total;
  tm.start(T);
  total.start(T);

  for (uint32_t p = threadIdx.x; p < MAX_FAN; p += THREADS) {
    S.cnt[p] = 0;
    S.cur[p] = NONE;
    S.fill[p] = CH;
    S.pend[p] = 0;
    S.pspill[p] = 0;
    S.hrec[p] = 0;
  }
  for (uint32_t i = threadIdx.x; i < cc.n; i += THREADS) {
    cc.key[i] = SKEY_EMPTY;
    cc.cnt[i] = 0;
    cc.sum[i] = 0;
    if (Ent<ENT>::MM) {
      cc.mn[i] = INT64_MAX;
      cc.mx[i] = INT64_MIN;
    }
  }
  if (threadIdx.x == 0) {
    S.first_spill = 1;
    S.tiles = 0;
    S.flush_tiles = 0;
    S.use_cache = cc.n != 0 && P.cache != 0;
    S.use_dedup = P.dedup;
    S.st_rows = S.st_hits = S.st_dups = 0;
  }
  __syncthreads();

  // ================= level 0: the input stream
  {
    Level L;
    L.level = 0;
    L.seed = level_seed(P.seed, 0);
    L.s_act = P.s_act0;
    L.dst = 0;
    L.fan_mask = fan - 1;
    // Tiles are claimed dynamically from a per-run counter, one iteration
    // ahead so that the next tile can be staged in L2 while this one runs.
    const uint64_t ntiles = (P.n + TILE - 1) / TILE;
    if (threadIdx.x == 0) S.tile_q[0] = atomicAdd(&C->tile_next, 1ull);
    adapt_begin_tile(S, cc.n != 0 && P.cache != 0, P.dedup != 0);
    for (uint32_t it = 0;; ++it) {
      // tile_q[it & 1] and this tile's feature flags are visible; every thread
      // is done with the previous tile
      __syncthreads();
      const uint64_t t = S.tile_q[it & 1];
      if (t >= ntiles) break;
      if (S.flush_tiles >= CACHE_FLUSH_TILES) cache_flush<ENT>(P, cc, S);
      const uint64_t row0 = t * TILE;
      if (threadIdx.x == 0) {
        const uint64_t nt = atomicAdd(&C->tile_next, 1ull);
        S.tile_q[(it + 1) & 1] = nt;
        if (P.vec_ok && !P.no_prefetch && nt < ntiles) {  // stage the next tile in L2
          const uint64_t nr0 = nt * TILE;
          const uint64_t nrows = P.n - nr0 < (uint64_t)TILE ? P.n - nr0 : (uint64_t)TILE;
          prefetch_l2(P.keys + nr0, (uint32_t)(nrows * 8));
          if (P.has_vals)
            prefetch_l2(static_cast<const char*>(P.vals) + nr0 * (VT == AGG_I64 ? 8 : 4),
                        (uint32_t)(nrows * (VT == AGG_I64 ? 8 : 4)));
        }
      }
      long long k[RPT], v[RPT];
      bool valid[RPT];
#pragma unroll
      for (int j = 0; j < RPT / 2; ++j) {
        const uint64_t row = row0 + (uint64_t)j * 2 * THREADS + 2 * threadIdx.x;
        if (P.vec_ok && row + 1 < P.n) {
          const longlong2 kk = __ldcs(reinterpret_cast<const longlong2*>(P.keys + row));
          k[2 * j] = kk.x;
          k[2 * j + 1] = kk.y;
          if (!P.has_vals) {
            v[2 * j] = v[2 * j + 1] = 0;
          } else if (VT == AGG_I64) {
            const longlong2 vv = __ldcs(reinterpret_cast<const longlong2*>(static_cast<const long long*>(P.vals) + row));
            v[2 * j] = vv.x;
            v[2 * j + 1] = vv.y;
          } else {
            const int2 vv = __ldcs(reinterpret_cast<const int2*>(static_cast<const int*>(P.vals) + row));
            v[2 * j] = vv.x;
            v[2 * j + 1] = vv.y;
          }
          valid[2 * j] = valid[2 * j + 1] = true;
        } else {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const uint64_t rr = row + e;
            valid[2 * j + e] = rr < P.n;
            k[2 * j + e] = 0;
            v[2 * j + e] = 0;
            if (rr < P.n) {
              k[2 * j + e] = __ldcs(reinterpret_cast<const long long*>(P.keys) + rr);
              if (P.has_vals)
                v[2 * j + e] = VT == AGG_I64 ? __ldcs(static_cast<const long long*>(P.vals) + rr)
                                             : (long long)__ldcs(static_cast<const int*>(P.vals) + rr);
            }
          }
        }
      }
      process_rows<ENT>(P, L, S, cc, k, v, valid, row0);
      adapt_end_tile(S, cc.n != 0 && P.cache != 0, P.dedup != 0);
      adapt_begin_tile(S, cc.n != 0 && P.cache != 0, P.dedup != 0);  // flags of the next tile
    }
    cache_flush<ENT>(P, cc, S);
    finalize_chunks(P, S, 0, 0);
    tm.lap(T, C, PH_L0);
    if (!grid_barrier(T, C, P.timeout_ns, S)) return RUN_ABORT;
    tm.lap(T, C, PH_L0_WAIT);
    const unsigned long long spilled = ld_relaxed_u64(&C->pool_next[0]);
    emit_table<ENT>(P, T, cc, L.s_act, 0, S);
    tm.lap(T, C, PH_L0_EMIT);
    if (spilled == 0) {
      total.lap(T, C, PH_TOTAL);
      final_step(P, T, 1);
      return RUN_DONE;
    }
    if (!grid_barrier(T, C, P.timeout_ns, S)) return RUN_ABORT;
    tm.lap(T, C, PH_ROUND_WAIT);
  }

  // ================= levels 1..: recursive processing of spilled partitions
  for (uint32_t level = 1;; ++level) {
    if (level >= AGG_MAX_LEVELS) {
      if (threadIdx.x == 0 && T.bid == 0) set_status(C, AGG_ERR_INTERNAL);
      final_step(P, T, level);
      return RUN_DONE;
    }
    const uint32_t src = (level + 1) & 1, dst = level & 1, set = level & 1;
    uint32_t* dpart = P.dir_part[src];
    uint32_t* dcount = P.dir_count[src];
    uint32_t* list = P.list[src];
    // P1: per-partition chunk and record counts of the source area.  Block 0
    // also clears the level's round counters here, before the level's first
    // barrier, so every block later reads the same values.
    if (threadIdx.x == 0 && T.bid == 0) {
      // Does this level fall back to sorting?  Every block reads the verdict
      // after the barrier below; the counters read here are final (the level
      // before ended with a barrier) and are reset only after this.
      uint32_t fb = 0;
      if (P.fallback_ok) {
        if (level >= P.max_levels) {
          fb = 1;
        } else {
          unsigned long long rows, groups;
          if (level == 1) {
            rows = P.n - C->spill_records[0];
            groups = C->resident_groups[0];
          } else {
            rows = C->lvl_sub_records[0] + C->lvl_sub_records[1];
            groups = C->lvl_sub_groups[0] + C->lvl_sub_groups[1];
          }
          if (rows > 0 && (double)groups > 0.8 * (double)rows) fb = 1;
        }
      }
      C->fallback_now = fb;
      C->pool_next[dst] = 0;
      C->overflow_used[level & 1] = 0;
      C->lvl_sub_records[0] = C->lvl_sub_records[1] = 0;
      C->lvl_sub_groups[0] = C->lvl_sub_groups[1] = 0;
    }
    // chunks handed out (a failed allocation still advanced the cursor)
    unsigned long long nch = ld_relaxed_u64(&C->pool_next[src]);
    if (nch > P.max_chunks[src]) nch = P.max_chunks[src];
    for (uint32_t p = threadIdx.x; p < MAX_FAN; p += THREADS) {
      S.cnt[p] = 0;
      S.hrec[p] = 0;
    }
    __syncthreads();
    for (unsigned long long c = T.bid * (unsigned long long)THREADS + threadIdx.x; c < nch;
         c += (unsigned long long)T.nb * THREADS) {
      const uint32_t p = __ldcg(dpart + c);
      atomicAdd(&S.cnt[p], 1u);
      smem_add_u64(&S.hrec[p], (unsigned long long)__ldcg(dcount + c));
    }
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < fan; p += THREADS) {
      if (S.cnt[p]) {
        atomicAdd(&C->part_chunks[set][p], S.cnt[p]);
        atomicAdd(&C->part_records[set][p], S.hrec[p]);
      }
      S.cnt[p] = 0;
    }
    if (!grid_barrier(T, C, P.timeout_ns, S)) return RUN_ABORT;
    if (ld_acquire_u32(&C->fallback_now)) {
      // every record of this level goes to the sort fallback (run by the
      // caller, so that its calls stay out of this function's hot loops)
      if (threadIdx.x == 0) {
        S.fb_level = level;
        S.fb_src = src;
        S.fb_dst = dst;
        S.fb_set = set;
        S.fb_nch = nch;
      }
      __syncthreads();
      return RUN_FALLBACK;
    }
    // P3: chunk lists grouped by partition
    if (threadIdx.x == 0) {
      uint32_t acc = 0;
      for (uint32_t p = 0; p < fan; ++p) {
        S.begin[p] = acc;
        acc += __ldcg(&C->part_chunks[set][p]);
      }
      S.begin[fan] = acc;
    }
    __syncthreads();
    for (unsigned long long c = T.bid * (unsigned long long)THREADS + threadIdx.x; c < nch;
         c += (unsigned long long)T.nb * THREADS) {
      const uint32_t p = __ldcg(dpart + c);
      const uint32_t at = atomicAdd(&C->part_cursor[set][p], 1u);
      list[S.begin[p] + at] = (uint32_t)c;
    }
    if (!grid_barrier(T, C, P.timeout_ns, S)) return RUN_ABORT;
    if (threadIdx.x == 0 && T.bid == 0) {
      for (uint32_t p = 0; p < MAX_FAN; ++p) {
        C->part_records[set ^ 1][p] = 0;
        C->part_chunks[set ^ 1][p] = 0;
        C->part_cursor[set ^ 1][p] = 0;
      }
    }
    tm.lap(T, C, PH_LISTS);
    // Rounds.  At levels >= 1 the global table keeps the first 1/GTABLE_DIV of the
    // slots (keys that overflow shared memory, partitions too big for a
    // shared-memory round) and the rest of the entry memory serves as
    // sub-partition scratch.  Whole partitions are packed into each round.
    const uint32_t gslots = (P.slots / GTABLE_DIV) / BUCKET * BUCKET;
    longlong2* scratch = reinterpret_cast<longlong2*>(P.ent + (size_t)gslots * Ent<ENT>::ES);
    // the per-block histogram rows of the shared-memory rounds sit at the end of the scratch
    const uint64_t scratch_bytes = (uint64_t)(P.slots - gslots) * Ent<ENT>::ES;
    // (at most a quarter of the scratch; fewer columns make larger sub-partitions)
    uint64_t hs = 2ull * cc.n < NSUB_MAX ? 2ull * cc.n : NSUB_MAX;
    const uint64_t hs_fit = scratch_bytes / 4 / ((uint64_t)T.nb * 4);
    if (hs > hs_fit) hs = hs_fit;
    const uint32_t hstride = hs > 0 ? (uint32_t)hs : 1u;
    const uint64_t hbytes = ((uint64_t)T.nb * hstride * 4 + 255) / 256 * 256;
    const uint64_t scratch_recs = scratch_bytes > hbytes ? (scratch_bytes - hbytes) / REC_BYTES : 0;
    uint32_t* hrows = reinterpret_cast<uint32_t*>(P.ent + (size_t)gslots * Ent<ENT>::ES + scratch_recs * REC_BYTES);
    const uint64_t round_cap = scratch_recs < ROUND_CAP_MAX ? scratch_recs : ROUND_CAP_MAX;
    const bool smem_ok = cc.n >= (uint32_t)THREADS && round_cap >= (uint64_t)TILE;
    Level G;
    G.level = level;
    G.seed = level_seed(P.seed, level);
    G.s_act = gslots;
    G.dst = dst;
    G.fan_mask = fan - 1;
    uint32_t rnd = 0;
    uint32_t p = 0;
    while (true) {
      while (p < fan && __ldcg(&C->part_records[set][p]) == 0) ++p;
      if (p >= fan) break;
      uint64_t tot = __ldcg(&C->part_records[set][p]);
      uint32_t q = p + 1;
      if (smem_ok && tot <= round_cap) {
        while (q < fan) {
          const uint64_t r = __ldcg(&C->part_records[set][q]);
          if (tot + r > round_cap || tot + r > ROUND_PACK_MAX) break;
          tot += r;
          ++q;
        }
        if (!smem_round<ENT>(P, T, tm, G, S, cc, src, S.begin[p], S.begin[q], tot, rnd & 1, scratch, hrows,
                                 hstride))
          return RUN_ABORT;
        if (threadIdx.x == 0 && T.bid == 0) C->rounds += 1;
        ++rnd;
        tm.lap(T, C, PH_ROUND_AGG);
        p = q;
        continue;
      }
      // a partition too big for a shared-memory round: global-table round
      const uint32_t c0 = S.begin[p], c1 = S.begin[q];
      const uint64_t ntiles = c1 - c0;
      if (!grid_barrier(T, C, P.timeout_ns, S)) return RUN_ABORT;  // shared-memory rounds before it are complete
      for (uint64_t t = T.bid; t < ntiles; t += T.nb) {
        if (threadIdx.x == 0 && t + T.nb < ntiles && !P.stg_host) {  // one tile is one chunk (CH == TILE)
          const uint32_t nc = __ldcg(list + c0 + (uint32_t)(t + T.nb));
          prefetch_l2(P.stg[src] + (size_t)nc * CH * REC_BYTES, __ldcg(dcount + nc) * (uint32_t)REC_BYTES);
        }
        adapt_begin_tile(S, cc.n != 0 && P.cache != 0, P.dedup != 0);
        __syncthreads();
        if (S.flush_tiles >= CACHE_FLUSH_TILES) cache_flush<ENT>(P, cc, S);
        long long k[RPT], v[RPT];
        bool valid[RPT];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          k[r] = 0;
          v[r] = 0;
          valid[r] = load_chunk_record(P, src, list, dcount, c0, t, r, k[r], v[r]);
        }
        process_rows<ENT>(P, G, S, cc, k, v, valid, 0);
        adapt_end_tile(S, cc.n != 0 && P.cache != 0, P.dedup != 0);
      }
      cache_flush<ENT>(P, cc, S);
      tm.lap(T, C, PH_ROUND_AGG);
      if (!grid_barrier(T, C, P.timeout_ns, S)) return RUN_ABORT;
      tm.lap(T, C, PH_ROUND_WAIT);
      emit_table<ENT>(P, T, cc, gslots, level, S);
      if (threadIdx.x == 0 && T.bid == 0) C->rounds += 1;
      tm.lap(T, C, PH_ROUND_EMIT);
      if (!grid_barrier(T, C, P.timeout_ns, S)) return RUN_ABORT;
      tm.lap(T, C, PH_ROUND_WAIT);
      p = q;
    }
    finalize_chunks(P, S, dst, level);
    if (!grid_barrier(T, C, P.timeout_ns, S)) return RUN_ABORT;
    tm.lap(T, C, PH_ROUND_WAIT);
    if (ld_acquire_u32(&C->overflow_used[level & 1])) emit_table<ENT>(P, T, cc, gslots, level, S);
    tm.lap(T, C, PH_ROUND_EMIT);
    if (ld_relaxed_u64(&C->pool_next[dst]) == 0) {
      restore_scratch<ENT>(P, T, gslots);
      total.lap(T, C, PH_TOTAL);
      final_step(P, T, level + 1);
      return RUN_DONE;
    }
  }
}

// The sort fallback of the level run_groupby stopped at (S.fb_*): sorts every
// record of the level and reduces them by segments, then finishes the run.
// False when a bounded wait gave up.
template <int ENT>
__device__ __noinline__ bool run_fallback(const HashParams& P, const Team& T, Smem& S, const Cache& cc) {
  Ctrl* C = P.ctrl;
  const uint32_t level = S.fb_level, src = S.fb_src, dst = S.fb_dst, set = S.fb_set;
  const unsigned long long nch = S.fb_nch;
  const uint32_t fan = 1u << P.fan_log2;
  unsigned long long recs = 0;
  for (uint32_t q = 0; q < fan; ++q) recs += __ldcg(&C->part_records[set][q]);
  if (recs >= (1ull << 32)) {  // beyond the sort's 32-bit offsets
    if (threadIdx.x == 0 && T.bid == 0) set_status(C, AGG_ERR_INTERNAL);
    final_step(P, T, level + 1);
    return true;
  }
  const uint32_t gsl = (P.slots / GTABLE_DIV) / BUCKET * BUCKET;
  uint32_t* H = reinterpret_cast<uint32_t*>(P.ent + (size_t)gsl * Ent<ENT>::ES);
  uint32_t* TOT = H + (size_t)T.nb * RADIX;
  longlong2* bufA = reinterpret_cast<longlong2*>(P.stg[dst]);
  longlong2* bufB = reinterpret_cast<longlong2*>(P.stg[src]);
  if (!fallback_sort(P, T, S, cc, src, nch, recs, bufA, bufB, H, TOT)) return false;
  const unsigned long long base = ld_relaxed_u64(&C->out_count);
  unsigned long long ng = 0;
  if (seg_reduce(P, T, S, RecordRows{bufB}, recs, false, base, &ng) < 0) return false;
  if (threadIdx.x == 0 && T.bid == 0) {
    C->out_count = base + ng;
    C->resident_groups[level] += ng;
    C->fallback_records = recs;
    C->fallback_level = level;
  }
  restore_scratch<ENT>(P, T, gsl);
  final_step(P, T, level + 1);
  return true;
}

template <int ENT, int VT>
__global__ void __launch_bounds__(THREADS, 2) hash_groupby_kernel(const __grid_constant__ HashParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const Cache cc = carve_cache(smem_raw + ((sizeof(Smem) + 15) & ~size_t(15)), P.ns, Ent<ENT>::MM);
  const Team T{gridDim.x, blockIdx.x};
  // sorted input: one segmented reduction, no table (falls through when unsorted)
  if (P.sorted_probe && P.n >= 2 && sorted_sample(P, S)) {
    Timer total;
    total.start(T);
    const int r = sorted_groupby<ENT, VT>(P, T, S);
    if (r < 0) return;
    if (r > 0) {
      total.lap(T, P.ctrl, PH_TOTAL);
      final_step(P, T, 1);
      return;
    }
  }
  if (run_groupby<ENT, VT>(P, T, S, cc) == RUN_FALLBACK) run_fallback<ENT>(P, T, S, cc);
}

// Batched group-by: teams of `team_blocks` consecutive blocks; team t runs the
// instances team_items[team_off[t] .. team_off[t+1]) one after another, each
// with the whole algorithm of run_groupby.  A team barrier between instances
// keeps a block from starting the next instance while another block of the
// team still finishes the previous one.
template <int ENT, int VT>
__global__ void __launch_bounds__(THREADS, 2)
    hash_batch_kernel(const HashParams* __restrict__ items, const uint32_t* __restrict__ team_off,
                      const uint32_t* __restrict__ team_items, uint32_t team_blocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const uint32_t team = blockIdx.x / team_blocks;
  const Team T{team_blocks, blockIdx.x % team_blocks};
  for (uint32_t j = team_off[team]; j < team_off[team + 1]; ++j) {
    const HashParams& P = items[team_items[j]];
    const Cache cc = carve_cache(smem_raw + ((sizeof(Smem) + 15) & ~size_t(15)), P.ns, Ent<ENT>::MM);
    int r = run_groupby<ENT, VT>(P, T, S, cc);
    if (r == RUN_FALLBACK) r = run_fallback<ENT>(P, T, S, cc) ? RUN_DONE : RUN_ABORT;
    if (r == RUN_ABORT) return;
    if (!grid_barrier(T, P.ctrl, P.timeout_ns, S)) return;
  }
}

// ---------------------------------------------------------------- in-budget fast path

// When a run has at most half as many rows as the table has slots, every
// distinct key fits in the table at once, and the whole group-by completes in
// place: a table that never fills needs no partitioning (Section 4.3.4).  Keys
// then probe linearly across all active slots instead of only their bucket, so
// no key is ever refused and nothing spills.  With no spill there is no phase to
// wait for: the aggregation runs as one ordinary launch with no grid barrier,
// and the emit as a second ordinary launch behind it in the stream.  Hot keys
// are absorbed by the per-block shared-memory cache as at level 0.

#ifndef AGG_FAST_RPT
#define AGG_FAST_RPT 8
#endif
#ifndef AGG_PART_ROWS_NUM
#define AGG_PART_ROWS_NUM 1
#endif
#ifndef AGG_PART_ROWS_DEN
#define AGG_PART_ROWS_DEN 1
#endif
#ifndef AGG_PART_DEDUP
#define AGG_PART_DEDUP 0
#endif
constexpr int FAST_RPT = AGG_FAST_RPT;                     // rows per thread of the aggregation pass
constexpr uint32_t FAST_ROWS = (uint32_t)THREADS * FAST_RPT;  // rows per block
constexpr int EMIT_THREADS = 256;
constexpr uint32_t EMIT_SLOTS = (uint32_t)EMIT_THREADS * 16;  // slots per emit block (16 tag bytes a thread)

// Home slot of a key among s_act slots (hash bits 32..63).
__device__ __forceinline__ uint32_t fast_home(uint64_t h, uint32_t s_act) {
  return (uint32_t)(((h >> 32) * (uint64_t)s_act) >> 32);
}

// Finds or claims the slot of `key` by linear probing from `slot` (its home),
// given the key word already loaded there (`k2`).  The table holds fewer
// distinct keys than s_act, so a probe always ends.  A claimed slot gets its
// tag byte, which marks it for the emit.
template <int ENT>
__device__ __forceinline__ uint32_t fast_probe(const HashParams& P, uint32_t s_act, long long key, uint64_t h,
                                               uint32_t slot, long long k2, bool* claimed = nullptr) {
  if (key == EMPTY_KEY) {  // the empty marker value itself: side slot
    uint8_t* tb = reinterpret_cast<uint8_t*>(P.tags) + P.slots;
    if (__ldcg(tb) == 0) __stcg(tb, (uint8_t)0x80);
    return P.slots;
  }
  for (;;) {
    if (k2 == key) return slot;
    if (k2 == EMPTY_KEY) {
      long long* kp = reinterpret_cast<long long*>(Ent<ENT>::at(P.ent, slot));
      const long long old = (long long)atomicCAS(reinterpret_cast<unsigned long long*>(kp),
                                                 (unsigned long long)EMPTY_KEY, (unsigned long long)key);
      if (old == EMPTY_KEY) {
        __stcg(reinterpret_cast<uint8_t*>(P.tags) + slot, (uint8_t)key_tag(h));
        if (claimed) *claimed = true;
        return slot;
      }
      if (old == key) return slot;
    }
    slot = slot + 1 == s_act ? 0u : slot + 1;
    k2 = __ldcg(reinterpret_cast<const long long*>(Ent<ENT>::at(P.ent, slot)));
  }
}

template <int ENT, int VT>
__global__ void __launch_bounds__(THREADS, 2) fast_agg_kernel(const HashParams P, uint32_t s_act) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const Cache cc = carve_cache(smem_raw + ((sizeof(Smem) + 15) & ~size_t(15)), P.cache ? P.ns : 0u, Ent<ENT>::MM);
  const uint64_t seed0 = level_seed(P.seed, 0);
  const uint64_t row0 = (uint64_t)blockIdx.x * FAST_ROWS;
  long long k[FAST_RPT], v[FAST_RPT];
  bool valid[FAST_RPT];
  // every load of the block's rows first
#pragma unroll
  for (int j = 0; j < FAST_RPT / 2; ++j) {
    const uint64_t row = row0 + (uint64_t)j * 2 * THREADS + 2 * threadIdx.x;
    if (P.vec_ok && row + 1 < P.n) {
      const longlong2 kk = __ldcs(reinterpret_cast<const longlong2*>(P.keys + row));
      k[2 * j] = kk.x;
      k[2 * j + 1] = kk.y;
      if (!P.has_vals) {
        v[2 * j] = v[2 * j + 1] = 0;
      } else if (VT == AGG_I64) {
        const longlong2 vv = __ldcs(reinterpret_cast<const longlong2*>(static_cast<const long long*>(P.vals) + row));
        v[2 * j] = vv.x;
        v[2 * j + 1] = vv.y;
      } else {
        const int2 vv = __ldcs(reinterpret_cast<const int2*>(static_cast<const int*>(P.vals) + row));
        v[2 * j] = vv.x;
        v[2 * j + 1] = vv.y;
      }
      valid[2 * j] = valid[2 * j + 1] = true;
    } else {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const uint64_t rr = row + e;
        valid[2 * j + e] = rr < P.n;
        k[2 * j + e] = 0;
        v[2 * j + e] = 0;
        if (rr < P.n) {
          k[2 * j + e] = __ldcs(reinterpret_cast<const long long*>(P.keys) + rr);
          if (P.has_vals)
            v[2 * j + e] = VT == AGG_I64 ? __ldcs(static_cast<const long long*>(P.vals) + rr)
                                         : (long long)__ldcs(static_cast<const int*>(P.vals) + rr);
        }
      }
    }
  }
  for (uint32_t i = threadIdx.x; i < cc.n; i += THREADS) {
    cc.key[i] = SKEY_EMPTY;
    cc.cnt[i] = 0;
    cc.sum[i] = 0;
    if (Ent<ENT>::MM) {
      cc.mn[i] = INT64_MAX;
      cc.mx[i] = INT64_MIN;
    }
  }
  __syncthreads();
  uint64_t h[FAST_RPT];
  bool need[FAST_RPT], cfree[FAST_RPT];
#pragma unroll
  for (int r = 0; r < FAST_RPT; ++r) {
    h[r] = fmix64((uint64_t)k[r] ^ seed0);
    cfree[r] = true;
    bool hit = false;
    if (valid[r]) hit = cache_hit<ENT>(cc, k[r], h[r], 1ull, (unsigned long long)v[r], v[r], v[r], cfree[r]);
    need[r] = valid[r] && !hit;
  }
  // key word at every remaining row's home slot, all loads in flight together
  uint32_t slot[FAST_RPT];
  long long kf[FAST_RPT];
#pragma unroll
  for (int r = 0; r < FAST_RPT; ++r) {
    slot[r] = fast_home(h[r], s_act);
    kf[r] = need[r] && k[r] != EMPTY_KEY ? __ldcg(reinterpret_cast<const long long*>(Ent<ENT>::at(P.ent, slot[r])))
                                         : EMPTY_KEY;
  }
#pragma unroll
  for (int r = 0; r < FAST_RPT; ++r) {
    if (!need[r]) continue;
    const uint32_t sl = fast_probe<ENT>(P, s_act, k[r], h[r], slot[r], kf[r]);
    Ent<ENT>::add(Ent<ENT>::at(P.ent, sl), P.ops, 1ull, (unsigned long long)v[r], v[r], v[r]);
    if (cfree[r]) cache_insert(cc, S, k[r], h[r], sl);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < cc.n; i += THREADS) {
    const long long key = cc.key[i];
    const unsigned long long c = cc.cnt[i];
    if (key == SKEY_EMPTY || c == 0) continue;
    Ent<ENT>::add(Ent<ENT>::at(P.ent, cc.slot[i]), P.ops, c, cc.sum[i], Ent<ENT>::MM ? cc.mn[i] : 0,
                  Ent<ENT>::MM ? cc.mx[i] : 0);
  }
}

// Emits every occupied slot among [0, s_act) (and the side slot), resetting
// each, then the last block to finish publishes the group count.  A thread
// reads 16 tag bytes; each warp reserves its output rows with one atomic.
template <int ENT>
__global__ void __launch_bounds__(EMIT_THREADS) fast_emit_kernel(const HashParams P, uint32_t s_act) {
  Ctrl* C = P.ctrl;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t words = s_act / 4;
  const uint64_t w0 = ((uint64_t)blockIdx.x * EMIT_THREADS + threadIdx.x) * 4;
  uint32_t tw[4] = {0u, 0u, 0u, 0u};
  if (w0 + 4 <= words) {
    const uint4 t = __ldcg(reinterpret_cast<const uint4*>(P.tags + w0));
    tw[0] = t.x;
    tw[1] = t.y;
    tw[2] = t.z;
    tw[3] = t.w;
  } else {
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) tw[q] = (w0 + q < words) ? __ldcg(P.tags + w0 + q) : 0u;
  }
  uint32_t oc = 0;
#pragma unroll
  for (uint32_t q = 0; q < 4; ++q) oc += __popc(~__vcmpeq4(tw[q], 0u) & 0x01010101u);
  uint32_t incl = oc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
    if ((int)lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && total) base = atomicAdd(&C->out_count, (unsigned long long)total);
  base = __shfl_sync(FULL_MASK, base, 31);
  unsigned long long pos = base + incl - oc;
#pragma unroll
  for (uint32_t q = 0; q < 4; ++q) {
    if (tw[q] == 0) continue;
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
      if (((tw[q] >> (8 * j)) & 0xFFu) == 0) continue;
      emit_one<ENT>(P, Ent<ENT>::at(P.ent, (uint32_t)(w0 + q) * 4 + j), pos);
      ++pos;
    }
    __stcg(P.tags + w0 + q, 0u);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // the side slot of the empty-marker key
    uint8_t* tb = reinterpret_cast<uint8_t*>(P.tags) + P.slots;
    if (__ldcg(tb)) {
      const unsigned long long at = atomicAdd(&C->out_count, 1ull);
      emit_one<ENT>(P, Ent<ENT>::at(P.ent, P.slots), at);
      __stcg(reinterpret_cast<long long*>(Ent<ENT>::at(P.ent, P.slots)), (long long)EMPTY_KEY);
      __stcg(tb, (uint8_t)0);
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  __threadfence();
  if (atomicAdd(&C->done_count, 1u) != gridDim.x - 1) return;
  __threadfence();
  volatile Ctrl* V = C;
  const unsigned long long ng = V->out_count;
  if (P.o_ngroups) *P.o_ngroups = ng;
  C->last_n_rows = P.n;
  C->last_n_groups = ng;
  C->last_levels = 1;
  C->last_rounds = 1;
  C->last_rows_at_full = ~0ull;
  for (int l = 0; l < AGG_MAX_LEVELS; ++l) {
    C->last_spill_records[l] = 0;
    C->last_resident_groups[l] = l == 0 ? ng : 0;
  }
  for (int ph = 0; ph < PHASES; ++ph) C->last_phase_ns[ph] = 0;
  C->last_sorted = 0;
  C->last_fallback_records = 0;
  C->last_fallback_level = 0;
  C->out_count = 0;
  __threadfence();
  C->done_count = 0;
}

// ---- partitioned in-budget path (small inputs): no global atomics
//
// For a small in-budget input the table's atomics, not memory, bound the pass
// (about four global atomics per row).  These inputs are therefore aggregated
// the way the hybrid hash aggregates partitions that fit in memory (Section
// 4.3), with a block's shared memory as that memory: the first launch splits
// each block's rows by the top hash bits into np partitions, a counting sort
// within the block written to a scratch area inside the budget (small enough
// to stay in L2); the second launch gives each partition to one block, which
// aggregates all of its records in its shared-memory table and writes its
// groups straight to the output.  Keys that do not fit a block's table go to
// the global table by linear probing (as in the fast path above), and the last
// block to finish emits that table when it was used, then publishes the count.

constexpr uint32_t PART_MAX = 2048;      // most partitions
constexpr uint32_t OVF_LIST = 65536;     // overflow-table slots listed for the last block (a scan past that)
constexpr uint32_t OVF_BLOCK = 2048;     // overflow-table slots a block lists and emits itself
constexpr uint32_t PART_MAX_BLK = 512;   // most first-launch blocks (2M rows)

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

// Exclusive scan over the block of one value per thread (THREADS threads).
__device__ __forceinline__ uint32_t block_scan_excl(uint32_t x, uint32_t* wsum, uint32_t& total) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL_MASK, inc, o);
    if ((int)lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t t = lane < WARPS ? wsum[lane] : 0u;
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL_MASK, ti, o);
      if ((int)lane >= o) ti += y;
    }
    if (lane < WARPS) wsum[lane] = ti - t;
    if (lane == WARPS - 1) wsum[WARPS] = ti;
  }
  __syncthreads();
  total = wsum[WARPS];
  const uint32_t r = wsum[warp] + inc - x;
  __syncthreads();
  return r;
}

// Launch 1: block b counting-sorts its FAST_ROWS rows by partition into
// rec[b * FAST_ROWS ...] and stores, for every partition q, its row count and
// start in the block's run at cnt[q * nblk + b] and start[q * nblk + b].
template <int VT>
__global__ void __launch_bounds__(THREADS, 2) part_scatter_kernel(const HashParams P, uint32_t plog, uint32_t nblk,
                                                               longlong2* __restrict__ rec, uint32_t* __restrict__ gcnt,
                                                               uint32_t* __restrict__ gstart) {
  __shared__ uint32_t cnt[PART_MAX];
  __shared__ uint32_t wsum[WARPS + 1];
  pdl_launch_dependents();  // the aggregation launch may start its set-up
  const uint32_t np = 1u << plog, b = blockIdx.x;
  const uint64_t row0 = (uint64_t)b * FAST_ROWS;
  const uint64_t seed0 = level_seed(P.seed, 0);
  long long k[FAST_RPT], v[FAST_RPT];
  bool valid[FAST_RPT];
#pragma unroll
  for (int j = 0; j < FAST_RPT / 2; ++j) {
    const uint64_t row = row0 + (uint64_t)j * 2 * THREADS + 2 * threadIdx.x;
    if (P.vec_ok && row + 1 < P.n) {
      const longlong2 kk = __ldcs(reinterpret_cast<const longlong2*>(P.keys + row));
      k[2 * j] = kk.x;
      k[2 * j + 1] = kk.y;
      if (!P.has_vals) {
        v[2 * j] = v[2 * j + 1] = 0;
      } else if (VT == AGG_I64) {
        const longlong2 vv = __ldcs(reinterpret_cast<const longlong2*>(static_cast<const long long*>(P.vals) + row));
        v[2 * j] = vv.x;
        v[2 * j + 1] = vv.y;
      } else {
        const int2 vv = __ldcs(reinterpret_cast<const int2*>(static_cast<const int*>(P.vals) + row));
        v[2 * j] = vv.x;
        v[2 * j + 1] = vv.y;
      }
      valid[2 * j] = valid[2 * j + 1] = true;
    } else {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const uint64_t rr = row + e;
        valid[2 * j + e] = rr < P.n;
        k[2 * j + e] = 0;
        v[2 * j + e] = 0;
        if (rr < P.n) {
          k[2 * j + e] = __ldcs(reinterpret_cast<const long long*>(P.keys) + rr);
          if (P.has_vals)
            v[2 * j + e] = VT == AGG_I64 ? __ldcs(static_cast<const long long*>(P.vals) + rr)
                                         : (long long)__ldcs(static_cast<const int*>(P.vals) + rr);
        }
      }
    }
  }
  for (uint32_t q = threadIdx.x; q < np; q += THREADS) cnt[q] = 0;
  __syncthreads();
  uint32_t part[FAST_RPT], rank[FAST_RPT];
#pragma unroll
  for (int r = 0; r < FAST_RPT; ++r) {
    part[r] = plog ? (uint32_t)(fmix64((uint64_t)k[r] ^ seed0) >> (64 - plog)) : 0u;
    rank[r] = valid[r] ? sh_atom_add_u32(&cnt[part[r]], 1u) : 0u;
  }
  __syncthreads();
  // partition starts within the block's run: exclusive scan over np counts
  const uint32_t per = (np + THREADS - 1) / THREADS, q0 = threadIdx.x * per;
  uint32_t mine = 0;
  for (uint32_t i = 0; i < per; ++i)
    if (q0 + i < np) mine += cnt[q0 + i];
  uint32_t total;
  uint32_t acc = block_scan_excl(mine, wsum, total);
  for (uint32_t i = 0; i < per; ++i) {
    const uint32_t q = q0 + i;
    if (q >= np) break;
    const uint32_t c = cnt[q];
    __stcg(gcnt + (size_t)q * nblk + b, c);
    __stcg(gstart + (size_t)q * nblk + b, acc);
    cnt[q] = acc;
    acc += c;
  }
  __syncthreads();
  longlong2* run = rec + (size_t)b * FAST_ROWS;
#pragma unroll
  for (int r = 0; r < FAST_RPT; ++r) {
    if (!valid[r]) continue;
    longlong2 x;
    x.x = k[r];
    x.y = v[r];
    __stcg(run + cnt[part[r]] + rank[r], x);
  }
}

// Emits the occupied slots of [0, s_act) with the whole block (rare: only
// when keys overflowed a block's shared-memory table).
template <int ENT>
__device__ void block_emit_table(const HashParams& P, uint32_t s_act) {
  Ctrl* C = P.ctrl;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t words = s_act / 4;
  for (uint32_t w0 = threadIdx.x * 4; w0 - threadIdx.x * 4 < words; w0 += THREADS * 4) {
    uint32_t tw[4];
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) tw[q] = (w0 + q < words) ? __ldcg(P.tags + w0 + q) : 0u;
    uint32_t oc = 0;
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) oc += __popc(~__vcmpeq4(tw[q], 0u) & 0x01010101u);
    uint32_t incl = oc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
      if ((int)lane >= o) incl += y;
    }
    const uint32_t tot = __shfl_sync(FULL_MASK, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && tot) base = atomicAdd(&C->out_count, (unsigned long long)tot);
    base = __shfl_sync(FULL_MASK, base, 31);
    unsigned long long pos = base + incl - oc;
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      if (tw[q] == 0) continue;
#pragma unroll
      for (uint32_t j = 0; j < 4; ++j) {
        if (((tw[q] >> (8 * j)) & 0xFFu) == 0) continue;
        emit_one<ENT>(P, Ent<ENT>::at(P.ent, (w0 + q) * 4 + j), pos);
        ++pos;
      }
      __stcg(P.tags + w0 + q, 0u);
    }
  }
}

// Launch 2: block q aggregates partition q.  Global table [0, s_ovf) takes the
// keys its shared-memory table cannot hold; the empty-marker key value takes
// the side slot.  The last block to finish emits those and publishes the run.
template <int ENT>
__global__ void __launch_bounds__(THREADS, 2)
    part_agg_kernel(const HashParams P, uint32_t plog, uint32_t nblk, const longlong2* __restrict__ rec,
                    const uint32_t* __restrict__ gcnt, const uint32_t* __restrict__ gstart, uint32_t s_ovf,
                    uint32_t* __restrict__ ovf_list) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t pre[PART_MAX_BLK + 1];
  __shared__ uint32_t sst[PART_MAX_BLK];
  __shared__ uint32_t wsum[WARPS + 1];
  __shared__ uint32_t last;
  // overflow-table slots this block claimed: every row of a key lies in one
  // partition, so only this block updates them and it emits them itself
  __shared__ uint32_t my_ovf[OVF_BLOCK];
  __shared__ uint32_t my_ovf_n;
  __shared__ unsigned long long my_ovf_base;
  Ctrl* C = P.ctrl;
  const Cache cc = carve_cache(smem_raw + ((sizeof(Smem) + 15) & ~size_t(15)), P.ns, Ent<ENT>::MM);
  const uint32_t q = blockIdx.x;
  if (threadIdx.x == 0) my_ovf_n = 0;
  const uint64_t seed0 = level_seed(P.seed, 0);
  for (uint32_t i = threadIdx.x; i < cc.n; i += THREADS) {
    cc.key[i] = SKEY_EMPTY;
    cc.cnt[i] = 0;
    cc.sum[i] = 0;
    if (Ent<ENT>::MM) {
      cc.mn[i] = INT64_MAX;
      cc.mx[i] = INT64_MIN;
    }
  }
  pdl_wait();  // the partitioning launch is complete and visible
  uint32_t c = 0;
  if (threadIdx.x < nblk) {
    c = __ldcg(gcnt + (size_t)q * nblk + threadIdx.x);
    sst[threadIdx.x] = __ldcg(gstart + (size_t)q * nblk + threadIdx.x);
  }
  uint32_t total;
  const uint32_t ex = block_scan_excl(c, wsum, total);  // nblk <= THREADS
  if (threadIdx.x < nblk) pre[threadIdx.x] = ex;
  if (threadIdx.x == 0) pre[nblk] = total;
  __syncthreads();
  bool ovf = false, side = false;
  constexpr int K = 4;
  for (uint32_t base = 0; base < total; base += THREADS * K) {
    long long k[K], v[K];
    bool in[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const uint32_t i = base + (uint32_t)j * THREADS + threadIdx.x;
      in[j] = i < total;
      k[j] = v[j] = 0;
      if (in[j]) {
        uint32_t lo = 0, hi = nblk;  // the run holding record i: pre[lo] <= i < pre[lo + 1]
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (pre[mid] <= i) lo = mid;
          else hi = mid;
        }
        const longlong2 x = __ldcg(rec + (size_t)lo * FAST_ROWS + sst[lo] + (i - pre[lo]));
        k[j] = x.x;
        v[j] = x.y;
      }
    }
#if AGG_PART_DEDUP
    // rows of equal keys in a warp are combined first: the lowest lane of each
    // key carries their partial state into the tables
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const uint32_t vm = __ballot_sync(FULL_MASK, in[j]);
      uint32_t peers = 0;
      if (in[j]) peers = __match_any_sync(vm, k[j]);
      const uint32_t leader = in[j] ? (uint32_t)__ffs(peers) - 1 : lane;
      const uint32_t gsize = __popc(peers);
      const uint32_t maxg = __reduce_max_sync(FULL_MASK, gsize);
      unsigned long long gs = (unsigned long long)v[j];
      long long gmn = v[j], gmx = v[j];
      uint32_t rem = (in[j] && lane == leader) ? (peers & ~(1u << lane)) : 0u;
      for (uint32_t it = 1; it < maxg; ++it) {
        const int src = rem ? __ffs(rem) - 1 : (int)lane;
        rem &= rem - 1;
        const long long ov = __shfl_sync(FULL_MASK, v[j], src);
        if (src != (int)lane) {
          gs += (unsigned long long)ov;
          gmn = ov < gmn ? ov : gmn;
          gmx = ov > gmx ? ov : gmx;
        }
      }
      if (!in[j] || lane != leader) continue;
      const uint64_t h = fmix64((uint64_t)k[j] ^ seed0);
      if (sub_upsert_part<ENT>(cc, k[j], h, gsize, gs, gmn, gmx)) continue;
      uint32_t sl = fast_home(h, s_ovf);
      const long long k2 =
          k[j] == EMPTY_KEY ? EMPTY_KEY : __ldcg(reinterpret_cast<const long long*>(Ent<ENT>::at(P.ent, sl)));
      bool claimed = false;
      sl = fast_probe<ENT>(P, s_ovf, k[j], h, sl, k2, &claimed);
      Ent<ENT>::add(Ent<ENT>::at(P.ent, sl), P.ops, gsize, gs, gmn, gmx);
      if (claimed) {
        const uint32_t mine = atomicAdd(&my_ovf_n, 1u);
        if (mine < OVF_BLOCK) {
          my_ovf[mine] = sl;
        } else {  // more than the block's list: the last block emits these
          const uint32_t at = atomicAdd(&C->ovf_listed, 1u);
          if (at < OVF_LIST) ovf_list[at] = sl;
          ovf = true;
        }
      }
      if (k[j] == EMPTY_KEY) side = true;
    }
#else
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (!in[j]) continue;
      const uint64_t h = fmix64((uint64_t)k[j] ^ seed0);
      if (sub_upsert<ENT>(cc, k[j], h, v[j])) continue;
      uint32_t sl = fast_home(h, s_ovf);
      const long long k2 =
          k[j] == EMPTY_KEY ? EMPTY_KEY : __ldcg(reinterpret_cast<const long long*>(Ent<ENT>::at(P.ent, sl)));
      bool claimed = false;
      sl = fast_probe<ENT>(P, s_ovf, k[j], h, sl, k2, &claimed);
      Ent<ENT>::add(Ent<ENT>::at(P.ent, sl), P.ops, 1ull, (unsigned long long)v[j], v[j], v[j]);
      if (claimed) {
        const uint32_t mine = atomicAdd(&my_ovf_n, 1u);
        if (mine < OVF_BLOCK) {
          my_ovf[mine] = sl;
        } else {  // more than the block's list: the last block emits these
          const uint32_t at = atomicAdd(&C->ovf_listed, 1u);
          if (at < OVF_LIST) ovf_list[at] = sl;
          ovf = true;
        }
      }
      if (k[j] == EMPTY_KEY) side = true;
    }
#endif
  }
  if (ovf) atomicOr(&C->overflow_used[0], 1u);
  if (side) atomicOr(&C->overflow_used[1], 1u);
  __syncthreads();
  sub_emit<ENT>(P, cc, 0);  // ends with a block barrier
  {
    const uint32_t m = my_ovf_n < OVF_BLOCK ? my_ovf_n : OVF_BLOCK;
    if (m) {  // this block's overflow keys are complete: emit them
      if (threadIdx.x == 0) {
        my_ovf_base = atomicAdd(&C->out_count, (unsigned long long)m);
        atomicAdd(&C->resident_groups[0], (unsigned long long)m);
      }
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < m; i += THREADS) {
        const uint32_t sl = my_ovf[i];
        emit_one<ENT>(P, Ent<ENT>::at(P.ent, sl), my_ovf_base + i);
        __stcg(reinterpret_cast<uint8_t*>(P.tags) + sl, (uint8_t)0);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&C->done_count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (ld_acquire_u32(&C->overflow_used[0])) {
    const uint32_t listed = ld_acquire_u32(&C->ovf_listed);
    if (listed <= OVF_LIST) {  // the claimed slots are listed: emit just those
      __shared__ unsigned long long list_base;
      if (threadIdx.x == 0) list_base = atomicAdd(&C->out_count, (unsigned long long)listed);
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < listed; i += THREADS) {
        const uint32_t sl = __ldcg(ovf_list + i);
        emit_one<ENT>(P, Ent<ENT>::at(P.ent, sl), list_base + i);
        __stcg(reinterpret_cast<uint8_t*>(P.tags) + sl, (uint8_t)0);
      }
    } else {
      block_emit_table<ENT>(P, s_ovf);
    }
  }
  if (threadIdx.x == 0 && ld_acquire_u32(&C->overflow_used[1])) {
    uint8_t* tb = reinterpret_cast<uint8_t*>(P.tags) + P.slots;
    if (__ldcg(tb)) {
      const unsigned long long at = atomicAdd(&C->out_count, 1ull);
      emit_one<ENT>(P, Ent<ENT>::at(P.ent, P.slots), at);
      __stcg(reinterpret_cast<long long*>(Ent<ENT>::at(P.ent, P.slots)), (long long)EMPTY_KEY);
      __stcg(tb, (uint8_t)0);
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  __threadfence();
  volatile Ctrl* V = C;
  const unsigned long long ng = V->out_count;
  if (P.o_ngroups) *P.o_ngroups = ng;
  C->last_n_rows = P.n;
  C->last_n_groups = ng;
  C->last_levels = 1;
  C->last_rounds = 1;
  C->last_rows_at_full = ~0ull;
  for (int l = 0; l < AGG_MAX_LEVELS; ++l) {
    C->last_spill_records[l] = 0;
    C->last_resident_groups[l] = l == 0 ? ng : 0;
    C->resident_groups[l] = 0;
  }
  for (int ph = 0; ph < PHASES; ++ph) C->last_phase_ns[ph] = 0;
  C->last_sorted = 0;
  C->last_fallback_records = 0;
  C->last_fallback_level = 0;
  C->overflow_used[0] = 0;
  C->overflow_used[1] = 0;
  C->ovf_listed = 0;
  C->out_count = 0;
  __threadfence();
  C->done_count = 0;
}

template <int ENT>
void* part_agg_ptr() {
  return reinterpret_cast<void*>(&part_agg_kernel<ENT>);
}

void* pick_part_agg(int ent) {
  if (ent == ENT32_CS) return part_agg_ptr<ENT32_CS>();
  if (ent == ENT32_CSMM32) return part_agg_ptr<ENT32_CSMM32>();
  return part_agg_ptr<ENT64>();
}

template <int ENT, int VT>
void* fast_kernel_ptr() {
  return reinterpret_cast<void*>(&fast_agg_kernel<ENT, VT>);
}

void* pick_fast_kernel(int ent, int vt) {
  if (vt == AGG_I32) {
    if (ent == ENT32_CS) return fast_kernel_ptr<ENT32_CS, AGG_I32>();
    if (ent == ENT32_CSMM32) return fast_kernel_ptr<ENT32_CSMM32, AGG_I32>();
    return fast_kernel_ptr<ENT64, AGG_I32>();
  }
  if (ent == ENT32_CS) return fast_kernel_ptr<ENT32_CS, AGG_I64>();
  return fast_kernel_ptr<ENT64, AGG_I64>();
}

template <int ENT>
__global__ void init_table_kernel(uint8_t* ent, uint32_t* tags, uint32_t slots) {
  // slots + 1 entries (the last is the side slot) and slots + BUCKET tag bytes
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s <= slots; s += (uint64_t)gridDim.x * blockDim.x) {
    Ent<ENT>::reset(Ent<ENT>::at(ent, (uint32_t)s));
  }
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < (slots + BUCKET) / 4;
       w += (uint64_t)gridDim.x * blockDim.x)
    tags[w] = 0;
}

template <int ENT>
__global__ void reset_entries_kernel(uint8_t* ent, uint64_t count) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < count; s += (uint64_t)gridDim.x * blockDim.x)
    Ent<ENT>::reset(Ent<ENT>::at(ent, (uint32_t)s));
}

template <int ENT, int VT>
void* kernel_ptr() {
  return reinterpret_cast<void*>(&hash_groupby_kernel<ENT, VT>);
}

template <int ENT, int VT>
void* batch_kernel_ptr() {
  return reinterpret_cast<void*>(&hash_batch_kernel<ENT, VT>);
}

void* pick_batch_kernel(int ent, int vt) {
  if (vt == AGG_I32) {
    if (ent == ENT32_CS) return batch_kernel_ptr<ENT32_CS, AGG_I32>();
    if (ent == ENT32_CSMM32) return batch_kernel_ptr<ENT32_CSMM32, AGG_I32>();
    return batch_kernel_ptr<ENT64, AGG_I32>();
  }
  if (ent == ENT32_CS) return batch_kernel_ptr<ENT32_CS, AGG_I64>();
  return batch_kernel_ptr<ENT64, AGG_I64>();
}

void* pick_kernel(int ent, int vt) {
  if (vt == AGG_I32) {
    if (ent == ENT32_CS) return kernel_ptr<ENT32_CS, AGG_I32>();
    if (ent == ENT32_CSMM32) return kernel_ptr<ENT32_CSMM32, AGG_I32>();
    return kernel_ptr<ENT64, AGG_I32>();
  }
  if (ent == ENT32_CS) return kernel_ptr<ENT32_CS, AGG_I64>();
  return kernel_ptr<ENT64, AGG_I64>();
}

size_t smem_bytes(int ent, uint32_t ns) {
  return ((sizeof(Smem) + 15) & ~size_t(15)) + cache_bytes(ns, ent != ENT32_CS);
}

}  // namespace

cudaError_t hash_kernel_info(int ent_kind, int vt, uint32_t ns, int device, KernelInfo* out) {
  void* k = pick_kernel(ent_kind, vt);
  const size_t smem = smem_bytes(ent_kind, ns);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(pick_fast_kernel(ent_kind, vt), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(pick_part_agg(ent_kind), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, THREADS, smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  out->blocks = per_sm * sms;
  out->smem = smem;
  return cudaSuccess;
}

cudaError_t hash_batch_kernel_info(int ent_kind, int vt, uint32_t ns, int device, KernelInfo* out) {
  void* k = pick_batch_kernel(ent_kind, vt);
  const size_t smem = smem_bytes(ent_kind, ns);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, THREADS, smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  out->blocks = per_sm * sms;
  out->smem = smem;
  return cudaSuccess;
}

cudaError_t hash_batch_launch(int ent_kind, int vt, const HashParams* items, const uint32_t* team_off,
                              const uint32_t* team_items, uint32_t team_blocks, uint32_t nteams, size_t smem,
                              cudaStream_t s) {
  void* k = pick_batch_kernel(ent_kind, vt);
  void* args[] = {const_cast<HashParams**>(&items), const_cast<uint32_t**>(&team_off),
                  const_cast<uint32_t**>(&team_items), &team_blocks};
  return cudaLaunchCooperativeKernel(k, dim3(nteams * team_blocks), dim3(THREADS), args, smem, s);
}

cudaError_t hash_launch(int ent_kind, int vt, const HashParams& p, const KernelInfo& ki, cudaStream_t s) {
  void* k = pick_kernel(ent_kind, vt);
  void* args[] = {const_cast<HashParams*>(&p)};
  return cudaLaunchCooperativeKernel(k, dim3(ki.blocks), dim3(THREADS), args, ki.smem, s);
}

void hash_fallback_plan(uint32_t fan, uint32_t max_levels, uint32_t blocks, uint64_t slots, uint32_t es, uint32_t ns,
                        bool staging, HashParams* p) {
  uint32_t bits = 0;
  while ((1u << bits) < fan) ++bits;
  // the levels of log2(fan)-bit digits that a sort-based split of 64-bit keys would need
  uint32_t cap = bits ? (64 + bits - 1) / bits : AGG_MAX_LEVELS - 1;
  if (cap > AGG_MAX_LEVELS - 1) cap = AGG_MAX_LEVELS - 1;
  if (max_levels) cap = max_levels;
  p->max_levels = cap;
  const uint64_t gslots = (slots / GTABLE_DIV) / BUCKET * BUCKET;
  const uint64_t scratch = (slots - gslots) * es;
  const uint64_t need = ((uint64_t)blocks * RADIX + RADIX) * 4 + 256;
  p->fallback_ok = staging && ns >= 512 && scratch >= need && blocks <= MAX_GRID ? 1u : 0u;
}

uint32_t hash_fast_slots(uint64_t n, uint64_t slots) {
  if (n > slots / 2) return 0;
  uint64_t a = 2 * n > MIN_SLOTS ? 2 * n : MIN_SLOTS;
  a = (a + BUCKET - 1) / BUCKET * BUCKET;
  return (uint32_t)(a < slots ? a : slots);
}

cudaError_t hash_fast_launch(int ent_kind, int vt, const HashParams& p, uint32_t s_act, size_t smem, cudaStream_t s) {
  if (p.n > 0) {
    const unsigned grid = (unsigned)((p.n + FAST_ROWS - 1) / FAST_ROWS);
    void* args[] = {const_cast<HashParams*>(&p), &s_act};
    const cudaError_t e = cudaLaunchKernel(pick_fast_kernel(ent_kind, vt), dim3(grid), dim3(THREADS), args, smem, s);
    if (e != cudaSuccess) return e;
  }
  const unsigned eg = (unsigned)((s_act + EMIT_SLOTS - 1) / EMIT_SLOTS);
  if (ent_kind == ENT32_CS) fast_emit_kernel<ENT32_CS><<<eg, EMIT_THREADS, 0, s>>>(p, s_act);
  else if (ent_kind == ENT32_CSMM32) fast_emit_kernel<ENT32_CSMM32><<<eg, EMIT_THREADS, 0, s>>>(p, s_act);
  else fast_emit_kernel<ENT64><<<eg, EMIT_THREADS, 0, s>>>(p, s_act);
  return cudaGetLastError();
}

#ifndef AGG_PART_OFF
#define AGG_PART_OFF 0
#endif
bool hash_part_plan(uint64_t n, uint64_t slots, uint32_t es, uint32_t ns, PartPlan* out) {
  if (AGG_PART_OFF || n == 0 || n > (uint64_t)PART_MAX_BLK * FAST_ROWS || ns < 256) return false;
  PartPlan pp;
  pp.nblk = (uint32_t)((n + FAST_ROWS - 1) / FAST_ROWS);
  uint32_t plog = 0;
  // rows per partition: about ns * AGG_PART_ROWS_NUM / AGG_PART_ROWS_DEN
  while ((1ull << plog) * ns * AGG_PART_ROWS_NUM < n * AGG_PART_ROWS_DEN && (1u << plog) < PART_MAX) ++plog;
  pp.plog = plog;
  uint64_t ovf = n + n / 4 > MIN_SLOTS ? n + n / 4 : MIN_SLOTS;  // at most n keys overflow: always room
  ovf = (ovf + BUCKET - 1) / BUCKET * BUCKET;
  pp.s_ovf = (uint32_t)ovf;
  const uint64_t rec_bytes = (uint64_t)pp.nblk * FAST_ROWS * 16;
  const uint64_t idx_bytes = 2ull * ((uint64_t)pp.nblk << plog) * 4 + (uint64_t)OVF_LIST * 4;
  const uint64_t scratch_slots = (rec_bytes + idx_bytes + 256 + es - 1) / es + 8;
  if (ovf + 1 + scratch_slots > slots) return false;  // the overflow table, then its side slot, stay clear
  pp.scratch_slot = (uint32_t)(slots - scratch_slots);  // scratch at the top of the entry memory
  *out = pp;
  return true;
}

cudaError_t hash_part_launch(int ent_kind, int vt, const HashParams& p, const PartPlan& pp, uint32_t es, size_t smem,
                             cudaStream_t s) {
  uint8_t* base = p.ent + (size_t)pp.scratch_slot * es;
  base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(base) + 255) & ~uintptr_t(255));
  longlong2* rec = reinterpret_cast<longlong2*>(base);
  uint32_t* gcnt = reinterpret_cast<uint32_t*>(base + (size_t)pp.nblk * FAST_ROWS * 16);
  uint32_t* gstart = gcnt + ((size_t)pp.nblk << pp.plog);
  uint32_t plog = pp.plog, nblk = pp.nblk, s_ovf = pp.s_ovf;
  if (vt == AGG_I32) part_scatter_kernel<AGG_I32><<<nblk, THREADS, 0, s>>>(p, plog, nblk, rec, gcnt, gstart);
  else part_scatter_kernel<AGG_I64><<<nblk, THREADS, 0, s>>>(p, plog, nblk, rec, gcnt, gstart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1u << plog);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const longlong2* crec = rec;
  const uint32_t* ccnt = gcnt;
  const uint32_t* cstart = gstart;
  uint32_t* olist = gstart + ((size_t)pp.nblk << pp.plog);
  void* args[] = {const_cast<HashParams*>(&p), &plog, &nblk, &crec, &ccnt, &cstart, &s_ovf, &olist};
  return cudaLaunchKernelExC(&cfg, pick_part_agg(ent_kind), args);
}

cudaError_t hash_reset_entries(uint8_t* ent, uint64_t count, int ent_kind, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((count + 255) / 256 > 4096 ? 4096 : (count + 255) / 256);
  if (ent_kind == ENT32_CS) reset_entries_kernel<ENT32_CS><<<blocks, 256, 0, s>>>(ent, count);
  else if (ent_kind == ENT32_CSMM32) reset_entries_kernel<ENT32_CSMM32><<<blocks, 256, 0, s>>>(ent, count);
  else reset_entries_kernel<ENT64><<<blocks, 256, 0, s>>>(ent, count);
  return cudaGetLastError();
}

cudaError_t hash_init_table(uint8_t* ent, uint32_t* tags, uint32_t slots, int ent_kind, cudaStream_t s) {
  const unsigned blocks = (unsigned)((slots + 255) / 256 > 4096 ? 4096 : (slots + 255) / 256 + 1);
  if (ent_kind == ENT32_CS) init_table_kernel<ENT32_CS><<<blocks, 256, 0, s>>>(ent, tags, slots);
  else if (ent_kind == ENT32_CSMM32) init_table_kernel<ENT32_CSMM32><<<blocks, 256, 0, s>>>(ent, tags, slots);
  else init_table_kernel<ENT64><<<blocks, 256, 0, s>>>(ent, tags, slots);
  return cudaGetLastError();
}

}  // namespace agg
