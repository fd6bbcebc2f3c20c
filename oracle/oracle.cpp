// CPU oracle for the budgeted group-by.  TEST INFRASTRUCTURE ONLY: it is used
// by tests/, by __graft_entry__.smoke() and by the cpu_baseline leg of bench.py,
// and never by the library's product path.  It shares no code, header, table or
// constant with the GPU path.
//
// What it computes (Section 3.1, "Aggregate Functions"): for every distinct
// grouping key k in keys[0..n), one group record (k, COUNT, SUM, MIN, MAX) whose
// grouping state aggregates the values of exactly the rows with key k.  These
// four bounded-state functions keep one fixed-size state per group (Section
// 3.1); AVG is the exact pair (SUM, COUNT).  SUM is taken modulo 2^64 (int64
// wrap-around), so it is associative and every algorithm reaches the same bits.
// Output records are sorted ascending by signed int64 key.
//
// oracle_groupby follows the memory discipline of the paper's Hash-Sort
// algorithm (Section 4.2): an in-memory hash map (std::unordered_map) holds
// group states until its estimated size would exceed the memory budget; then
// its groups are sorted by key, written out as one sorted run, and the map is
// emptied (phase 1).  At the end the runs and the final map are merged in key
// order and records with equal keys are combined (phase 2).  Runs sort on the
// key alone rather than on (slot id, key): the order inside a run does not
// change the result.
//
// oracle_groupby_bruteforce is the nested-loop definition for tiny inputs, and
// oracle_groups_of recomputes chosen groups by a full scan, for sampled checks
// at sizes where a full oracle run would take too long.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <functional>
#include <queue>
#include <unordered_map>
#include <utility>
#include <vector>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

namespace {

struct State {
  uint64_t count;
  uint64_t sum;  // two's-complement sum modulo 2^64
  int64_t min;
  int64_t max;
};

inline State first_state(int64_t v) {
  State s;
#if ORACLE_MUTANT == 5
  s.count = 0;  // planted: the first row of a group is not counted
#else
  s.count = 1;
#endif
  s.sum = (uint64_t)v;
#if ORACLE_MUTANT == 8
  s.min = 0;  // planted: MIN starts from 0 instead of the first value
#else
  s.min = v;
#endif
  s.max = v;
  return s;
}

inline void add_row(State& s, int64_t v) {
  s.count += 1;
#if ORACLE_MUTANT == 6
  s.sum = (uint64_t)(int64_t)(int32_t)(s.sum + (uint64_t)v);  // planted: 32-bit accumulator
#else
  s.sum += (uint64_t)v;
#endif
#if ORACLE_MUTANT == 2
  if (v > s.min) s.min = v;  // planted: MIN and MAX swapped
  if (v < s.max) s.max = v;
#else
  if (v < s.min) s.min = v;
  if (v > s.max) s.max = v;
#endif
}

inline void combine(State& a, const State& b) {
  a.count += b.count;
  a.sum += b.sum;
  if (b.min < a.min) a.min = b.min;
  if (b.max > a.max) a.max = b.max;
}

using Run = std::vector<std::pair<int64_t, State>>;

bool key_less(int64_t a, int64_t b) {
#if ORACLE_MUTANT == 4
  return (uint64_t)a < (uint64_t)b;  // planted: unsigned key order
#else
  return a < b;
#endif
}

Run sorted_run(const std::unordered_map<int64_t, State>& m) {
  Run r(m.begin(), m.end());
  std::sort(r.begin(), r.end(), [](const auto& x, const auto& y) { return key_less(x.first, y.first); });
  return r;
}

struct Out {
  int64_t* keys;
  uint64_t* count;
  int64_t* sum;
  int64_t* min;
  int64_t* max;
  uint64_t capacity;
  uint64_t n;
  bool overflow;
  void put(int64_t k, const State& s) {
    if (n >= capacity) {
      overflow = true;
      return;
    }
    if (keys) keys[n] = k;
    if (count) count[n] = s.count;
    if (sum) sum[n] = (int64_t)s.sum;
    if (min) min[n] = s.min;
    if (max) max[n] = s.max;
    ++n;
  }
};

}  // namespace

extern "C" {

// Budgeted group-by (Hash-Sort discipline, Section 4.2).  vals may be NULL
// (every value is then taken as 0).  entry_bytes is the memory charged per
// group held in the map; budget_bytes must allow at least one group.
// Returns 0 on success, 1 if out_capacity is too small, 2 on bad arguments.
int oracle_groupby(const int64_t* keys, const int64_t* vals, uint64_t n, uint64_t budget_bytes,
                   uint64_t entry_bytes, int64_t* out_keys, uint64_t* out_count, int64_t* out_sum,
                   int64_t* out_min, int64_t* out_max, uint64_t out_capacity, uint64_t* n_groups,
                   uint64_t* n_runs) {
  if ((n > 0 && keys == nullptr) || entry_bytes == 0 || budget_bytes < entry_bytes) return 2;
  const uint64_t max_groups = budget_bytes / entry_bytes;
  std::unordered_map<int64_t, State> table;
  std::vector<Run> runs;
#if ORACLE_MUTANT == 1
  const uint64_t last = n > 0 ? n - 1 : 0;  // planted: the last row is dropped
#else
  const uint64_t last = n;
#endif
  for (uint64_t i = 0; i < last; ++i) {
    const int64_t k = keys[i];
    const int64_t v = vals ? vals[i] : 0;
    auto it = table.find(k);
    if (it != table.end()) {
      add_row(it->second, v);
      continue;
    }
    if (table.size() + 1 > max_groups) {  // full: flush a sorted run, empty the table
      runs.push_back(sorted_run(table));
      table.clear();
    }
    table.emplace(k, first_state(v));
  }
#if ORACLE_MUTANT != 7
  if (!table.empty()) runs.push_back(sorted_run(table));  // (mutant 7 drops the final table)
#endif
  table.clear();

  // Phase 2: merge all runs in key order, combining equal keys.
  Out out{out_keys, out_count, out_sum, out_min, out_max, out_capacity, 0, false};
  using Head = std::pair<int64_t, size_t>;  // (key, run index)
  auto heap_after = [](const Head& a, const Head& b) { return key_less(b.first, a.first); };
  std::priority_queue<Head, std::vector<Head>, decltype(heap_after)> heap(heap_after);
  std::vector<size_t> pos(runs.size(), 0);
  for (size_t r = 0; r < runs.size(); ++r)
    if (!runs[r].empty()) heap.push({runs[r][0].first, r});
  bool have = false;
  int64_t cur_key = 0;
  State cur{};
  while (!heap.empty()) {
    const size_t r = heap.top().second;
    heap.pop();
    const auto& rec = runs[r][pos[r]];
#if ORACLE_MUTANT == 3
    if (have) out.put(cur_key, cur);  // planted: equal keys from different runs are not combined
    cur_key = rec.first;
    cur = rec.second;
    have = true;
#else
    if (have && rec.first == cur_key) {
      combine(cur, rec.second);
    } else {
      if (have) out.put(cur_key, cur);
      cur_key = rec.first;
      cur = rec.second;
      have = true;
    }
#endif
    if (++pos[r] < runs[r].size()) heap.push({runs[r][pos[r]].first, r});
  }
  if (have) out.put(cur_key, cur);
  if (n_groups) *n_groups = out.n;
  if (n_runs) *n_runs = runs.size();
  return out.overflow ? 1 : 0;
}

// Nested-loop definition: row i opens a group iff no earlier row has its key;
// the group then scans every row.  O(n^2): tiny inputs only.  Output sorted by
// key with an insertion sort.  Same return codes as oracle_groupby.
int oracle_groupby_bruteforce(const int64_t* keys, const int64_t* vals, uint64_t n, int64_t* out_keys,
                              uint64_t* out_count, int64_t* out_sum, int64_t* out_min, int64_t* out_max,
                              uint64_t out_capacity, uint64_t* n_groups) {
  if (n > 0 && keys == nullptr) return 2;
  std::vector<std::pair<int64_t, State>> groups;
  for (uint64_t i = 0; i < n; ++i) {
    bool seen = false;
    for (uint64_t j = 0; j < i; ++j)
      if (keys[j] == keys[i]) {
        seen = true;
        break;
      }
    if (seen) continue;
    State s{0, 0, 0, 0};
    bool first = true;
    for (uint64_t j = 0; j < n; ++j) {
      if (keys[j] != keys[i]) continue;
      const int64_t v = vals ? vals[j] : 0;
      if (first) {
        s = State{1, (uint64_t)v, v, v};
        first = false;
      } else {
        s.count += 1;
        s.sum += (uint64_t)v;
        s.min = v < s.min ? v : s.min;
        s.max = v > s.max ? v : s.max;
      }
    }
    // insertion into the key-sorted list
    size_t at = groups.size();
    groups.push_back({keys[i], s});
    while (at > 0 && groups[at - 1].first > groups[at].first) {
      std::swap(groups[at - 1], groups[at]);
      --at;
    }
  }
  Out out{out_keys, out_count, out_sum, out_min, out_max, out_capacity, 0, false};
  for (const auto& g : groups) out.put(g.first, g.second);
  if (n_groups) *n_groups = out.n;
  return out.overflow ? 1 : 0;
}

// Recomputes the groups of m chosen keys by one full scan of the input.
// A key that does not occur gets count 0, sum 0, min INT64_MAX, max INT64_MIN.
int oracle_groups_of(const int64_t* keys, const int64_t* vals, uint64_t n, const int64_t* sample, uint64_t m,
                     uint64_t* out_count, int64_t* out_sum, int64_t* out_min, int64_t* out_max) {
  if ((n > 0 && keys == nullptr) || (m > 0 && sample == nullptr)) return 2;
  std::vector<std::pair<int64_t, uint64_t>> order(m);
  for (uint64_t j = 0; j < m; ++j) order[j] = {sample[j], j};
  std::sort(order.begin(), order.end());
  std::vector<int64_t> sk(m);
  for (uint64_t j = 0; j < m; ++j) sk[j] = order[j].first;
  std::vector<State> st(m, State{0, 0, INT64_MAX, INT64_MIN});
  for (uint64_t i = 0; i < n; ++i) {
    auto it = std::lower_bound(sk.begin(), sk.end(), keys[i]);
    if (it == sk.end() || *it != keys[i]) continue;
    State& s = st[it - sk.begin()];
    const int64_t v = vals ? vals[i] : 0;
    s.count += 1;
    s.sum += (uint64_t)v;
    if (v < s.min) s.min = v;
    if (v > s.max) s.max = v;
  }
  for (uint64_t j = 0; j < m; ++j) {
    // equal sample keys share one state; copy it to every position
    const uint64_t src = std::lower_bound(sk.begin(), sk.end(), order[j].first) - sk.begin();
    const uint64_t dst = order[j].second;
    if (out_count) out_count[dst] = st[src].count;
    if (out_sum) out_sum[dst] = (int64_t)st[src].sum;
    if (out_min) out_min[dst] = st[src].min;
    if (out_max) out_max[dst] = st[src].max;
  }
  return 0;
}

// Number of distinct keys, by sorting a copy and counting key changes.
uint64_t oracle_count_distinct(const int64_t* keys, uint64_t n) {
  if (n == 0) return 0;
  std::vector<int64_t> k(keys, keys + n);
  std::sort(k.begin(), k.end());
  return (uint64_t)(std::unique(k.begin(), k.end()) - k.begin());
}

}  // extern "C"
