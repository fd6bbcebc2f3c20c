// Sort path of the budgeted group-by (Section 4.1): radix sort + segmented reduction.
#pragma once

#include "agg_internal.cuh"

namespace agg {

struct SortState {
  void* mem = nullptr;       // staging of the MSD partitions (outside the budget)
  uint64_t mem_bytes = 0;
  void* work = nullptr;      // double buffers + histograms (inside the budget)
  uint64_t work_bytes = 0;
  uint64_t reserved_rows = 0;
  uint64_t round_rows = 0;   // records sorted per round (fits the budget)
  uint32_t epoch = 0;        // look-back status epoch, one per pass
  uint64_t last_buckets = 0;
  uint64_t last_passes = 0;
  uint64_t last_rounds = 0;
  uint64_t last_levels = 0;
  uint64_t launches = 0;
  bool external = false;     // work lies in memory the caller owns (the hash table's, for AGG_PATH_AUTO)
};

agg_status sort_reserve(SortState& s, uint64_t rows, size_t budget, const agg_spec& spec);
agg_status sort_run(SortState& s, size_t budget, const agg_spec& spec, Ctrl* ctrl, const int64_t* d_keys,
                    const void* d_vals, uint64_t n, const agg_output* out, cudaStream_t stream);
void sort_free(SortState& s);
// Records one round can sort in work_bytes of working memory.
uint64_t sort_rows_for(uint64_t work_bytes);
// Uses caller-owned working memory (work_bytes at work) from now on; nothing is
// allocated for it and its look-back words are cleared before every run.
void sort_attach(SortState& s, void* work, uint64_t work_bytes);
uint64_t sort_staging_bytes(const SortState& s);
void sort_fill_stats(const SortState& s, agg_stats* st);
inline uint64_t sort_launches(const SortState& s) { return s.launches; }

}  // namespace agg
