// Sort path of the budgeted group-by (Section 4.1).
#include "sort_path.cuh"

namespace agg {

agg_status sort_reserve(SortState&, uint64_t, size_t, const agg_spec&) { return AGG_OK; }
agg_status sort_run(SortState&, size_t, const agg_spec&, Ctrl*, const int64_t*, const void*, uint64_t,
                    const agg_output*, cudaStream_t) {
  return AGG_ERR_INTERNAL;
}
void sort_free(SortState& s) {
  if (s.mem) cudaFree(s.mem);
  if (s.work) cudaFree(s.work);
  s = SortState{};
}
uint64_t sort_staging_bytes(const SortState& s) { return s.mem_bytes; }
void sort_fill_stats(const SortState&, agg_stats*) {}

}  // namespace agg
