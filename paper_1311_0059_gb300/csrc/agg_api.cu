// C ABI of libagg.so: handle lifetime, planning, staging reservation, runs.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <unordered_map>
#include <queue>
#include <vector>

#include "agg_internal.cuh"
#include "sort_path.cuh"

using namespace agg;

struct agg_handle {
  int device = 0;
  size_t budget = 0;
  agg_spec spec{};
  agg_tuning tune{};
  int ent_kind = 0;
  uint32_t es = 32;
  uint64_t slots = 0;
  uint64_t working_bytes = 0;
  // working memory (inside the budget)
  void* work = nullptr;
  Ctrl* ctrl = nullptr;
  uint32_t* tags = nullptr;
  uint8_t* ent = nullptr;
  KernelInfo ki{};
  // staging (outside the budget)
  void* stg_mem[2] = {nullptr, nullptr};
  uint8_t* stg[2] = {nullptr, nullptr};
  uint32_t* dir_part[2] = {nullptr, nullptr};
  uint32_t* dir_count[2] = {nullptr, nullptr};
  uint32_t* list[2] = {nullptr, nullptr};
  uint64_t max_chunks = 0;
  uint64_t reserved_rows = 0;
  uint32_t reserved_fan = 0;
  uint64_t staging_bytes = 0;
  bool stg_host = false;  // staging areas in pinned host memory
  // device copies for agg_run_host
  void* in_buf = nullptr;
  uint64_t in_cap = 0;
  void* out_buf = nullptr;
  uint64_t out_cap = 0;
  uint64_t* ng_host = nullptr;  // pinned
  // sort path working state
  SortState sort{};
  cudaStream_t last_stream = nullptr;
  bool ran = false;
  uint64_t launches = 0;
  // entries [dirty_lo, slots) hold scratch records of the partitioned in-budget
  // path (slots = none); they are restored before another run needs them
  uint64_t dirty_lo = 0;
  bool table_dirty = false;  // AGG_PATH_AUTO: a sort run used the table's memory
  int last_path = 0;         // path of the last run
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

constexpr double DEFAULT_LF = 0.5;
constexpr uint32_t DEFAULT_NS = 2048;
constexpr double DEFAULT_FUDGE = 1.2;
constexpr uint64_t TIMEOUT_NS = 4000000000ull;
constexpr uint32_t MAX_WAIT_LIMIT_US = 60000000u;  // a stuck run holds the GPU for at most a minute

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool valid_spec(const agg_spec* s) {
  if (!s) return false;
  if (s->ops == 0 || (s->ops & ~15u)) return false;
  if (s->value_type != AGG_I32 && s->value_type != AGG_I64) return false;
  if (s->path != AGG_PATH_HASH && s->path != AGG_PATH_SORT && s->path != AGG_PATH_AUTO) return false;
  if (s->flags != 0) return false;
  return true;
}

int pick_ent(const agg_spec* s) {
  if ((s->ops & (AGG_MIN | AGG_MAX)) == 0) return ENT32_CS;
  return s->value_type == AGG_I32 ? ENT32_CSMM32 : ENT64;
}

agg_tuning effective(const agg_tuning* t) {
  agg_tuning e{};
  e.max_load_factor = (t && t->max_load_factor > 0) ? t->max_load_factor : DEFAULT_LF;
  e.smem_entries = (t && t->smem_entries) ? t->smem_entries : DEFAULT_NS;
  e.fan_out = t ? t->fan_out : 0;
  e.warp_dedup = (t && t->warp_dedup) ? t->warp_dedup : 2;  // off unless asked for
  e.fudge = (t && t->fudge > 0) ? t->fudge : DEFAULT_FUDGE;
  e.wait_limit_us = t ? t->wait_limit_us : 0;
  e.in_budget = (t && t->in_budget) ? t->in_budget : 1;  // on unless asked off
  e.sorted_input = (t && t->sorted_input) ? t->sorted_input : 1;
  e.max_levels = t ? t->max_levels : 0;
  e.staging_tier = t ? t->staging_tier : 0;
  e.level0_slots = t ? t->level0_slots : 0;
  return e;
}

// Most slots the level-0 table may use (agg_tuning.level0_slots).
uint64_t level0_cap(const agg_tuning& e) {
  if (e.level0_slots == 0) return AGG_LEVEL0_SLOTS;
  if (e.level0_slots == 1) return ~0ull;
  return e.level0_slots;
}

bool valid_tuning(const agg_tuning* t) {
  if (!t) return true;
  if (t->max_load_factor < 0 || t->max_load_factor > 0.95) return false;
  if (t->smem_entries > 1) {
    if (t->smem_entries < 256 || t->smem_entries > 4096 || (t->smem_entries & (t->smem_entries - 1))) return false;
  }
  if (t->fan_out && (t->fan_out < 16 || t->fan_out > 256 || (t->fan_out & (t->fan_out - 1)))) return false;
  if (t->warp_dedup > 2) return false;
  if (t->wait_limit_us > MAX_WAIT_LIMIT_US) return false;
  if (t->fudge < 0 || t->fudge > 16) return false;
  if (t->in_budget > 2 || t->sorted_input > 2 || t->staging_tier > 2) return false;
  if (t->max_levels >= AGG_MAX_LEVELS) return false;
  if (t->level0_slots > 1 && t->level0_slots < MIN_SLOTS) return false;
  return true;
}

uint32_t next_pow2(uint64_t x) {
  uint32_t p = 1;
  while (p < x && p < (1u << 30)) p <<= 1;
  return p;
}

// Fan-out of the spill partitioning.  Eq. 1 (Section 4.3) gives the spilled
// partitions P = (G*F - M)/(M - 2) for a budget of M frames; with a frame-free
// byte budget M >> 2 this is P ~ G*F/M - 1 (G and M in bytes), the count that
// lets every spilled partition be aggregated within the budget next level.
// G is the result size: expected_groups if given, else n (an upper bound).
uint32_t plan_fan(const agg_spec* s, const agg_tuning& t, uint64_t n, size_t budget, uint32_t es) {
  if (t.fan_out) return t.fan_out;
  const double g = (double)(s->expected_groups ? s->expected_groups : n);
  const double p = g * (double)es * t.fudge / (double)budget;
  uint64_t want = (uint64_t)std::ceil(p > 1 ? p : 1);
  uint32_t f = next_pow2(want);
  if (f < 16) f = 16;
  if (f > 256) f = 256;
  return f;
}

uint32_t log2u(uint32_t x) {
  uint32_t l = 0;
  while ((1u << l) < x) ++l;
  return l;
}

struct Layout {
  uint64_t ctrl_bytes, tags_off, ent_off, slots, total;
};

// Working memory: [control block][tag bytes: S + BUCKET][entries: S + 1].
// Entry S is the side slot of the key value that marks empty slots.
bool layout_for(size_t budget, uint32_t es, Layout* L) {
  L->ctrl_bytes = align_up(sizeof(Ctrl), 256);
  if (budget < AGG_MIN_BUDGET) return false;
  const uint64_t fixed = L->ctrl_bytes + BUCKET + es + 512;
  uint64_t s = (budget - fixed) / (es + 1);
  s -= s % BUCKET;
  if (s > (1ull << 31) - BUCKET) s = (1ull << 31) - BUCKET;
  L->slots = s;
  L->tags_off = L->ctrl_bytes;
  L->ent_off = align_up(L->tags_off + s + BUCKET, 256);
  L->total = L->ent_off + (s + 1) * es;
  return s >= MIN_SLOTS && L->total <= budget;
}

uint32_t active_slots(uint64_t est, double lf, uint64_t slots, uint64_t cap = ~0ull) {
  uint64_t want = (uint64_t)((double)est / lf) + BUCKET;
  want = (want + BUCKET - 1) / BUCKET * BUCKET;
  if (want < MIN_SLOTS) want = MIN_SLOTS;
  if (want > cap) want = cap / BUCKET * BUCKET;
  if (want > slots) want = slots;
  return (uint32_t)want;
}

// ---- cost model of the two paths (Section 5's models, counted in DRAM bytes)
//
// Hash path: the input once; when the rows may not all fit the table
// (n > slots / 2), the Pre-Partitioning spill R(1 - K/G) of Section 5.3.4,
// written and read back once (the recursion completes at level 1 when its
// partitions fit the rounds); when the groups are more than 0.8 of the rows the
// spilled records are sorted at level 1 instead (eight radix passes, each
// reading and writing 16-byte records, then a reduction pass); the result.
// Sort path: a split pass when the rows exceed one round, the eight passes over
// (key, value), a reduction pass, the result.  Times are bytes over the
// effective bandwidth each path reached on GB300 (spilling workload: hash
// 10.9 GB in 12.4 ms, sort about 62 GB in 38.5 ms) plus a fixed cost per run.
constexpr double HASH_GBS = 880.0, SORT_GBS = 1620.0, INBUDGET_GBS = 300.0;
constexpr double HASH_FIXED_S = 30e-6, SORT_FIXED_S = 120e-6;

struct PathCosts {
  double hash_bytes, sort_bytes, hash_s, sort_s;
  int choice;  // AGG_PATH_HASH or AGG_PATH_SORT
};

PathCosts path_costs(const agg_spec* s, const agg_tuning& t, uint64_t n, size_t budget, uint32_t es,
                     uint64_t slots) {
  PathCosts c{};
  const double vb = s->value_type == AGG_I64 ? 8.0 : 4.0;
  const double rows = (double)n;
  const double g = s->expected_groups ? std::min((double)s->expected_groups, rows) : rows;
  const double out = g * 8.0 * (1 + __builtin_popcount(s->ops & 15u));
  const double in = rows * (8.0 + vb);
  // the level-0 table's planned groups (K)
  const double k = t.max_load_factor * (double)std::min<uint64_t>(slots, level0_cap(t));
  if (n <= slots / 2) {
    c.hash_bytes = in + out;
    c.hash_s = c.hash_bytes / (INBUDGET_GBS * 1e9) + HASH_FIXED_S;
  } else {
    const double spill = g > k ? rows * (1.0 - k / g) : 0.0;  // R(1 - K/G)
    double bytes = in + 2.0 * 16.0 * spill + out;
    if (g > 0.8 * rows) bytes += spill * (8.0 * 32.0 + 16.0);  // level 1 sorts instead
    c.hash_bytes = bytes;
    c.hash_s = bytes / (HASH_GBS * 1e9) + HASH_FIXED_S;
  }
  const uint64_t ctrl = align_up(sizeof(Ctrl), 256);
  const uint64_t rr = sort_rows_for(budget > ctrl ? budget - ctrl : 0);
  c.sort_bytes = (n > rr ? 2.0 * (8.0 + vb) * rows : 0.0) + 8.0 * rows + 8.0 * 32.0 * rows + 16.0 * rows + out;
  c.sort_s = c.sort_bytes / (SORT_GBS * 1e9) + SORT_FIXED_S;
  // with no estimate of G the model has nothing to go on: the hash path
  c.choice = s->expected_groups && c.sort_s < c.hash_s ? AGG_PATH_SORT : AGG_PATH_HASH;
  return c;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Checks the pointers of one group-by's input and output: device memory the
// kernel can address (so that a misplaced host pointer is an argument error,
// not a device fault), values present when an aggregate needs them, and keys
// and values aligned to their element size.  d_n_groups is checked only where
// the call uses it.
agg_status check_device_io(uint32_t ops, int32_t value_type, const int64_t* d_keys, const void* d_vals, uint64_t n,
                           const agg_output* out, bool uses_d_n_groups) {
  const bool need_vals = (ops & ~(uint32_t)AGG_COUNT) != 0;
  if (n > 0) {
    if (!is_device_ptr(d_keys)) return AGG_ERR_INVALID_ARG;
    if (need_vals && !is_device_ptr(d_vals)) return AGG_ERR_INVALID_ARG;
    if (d_vals && !is_device_ptr(d_vals)) return AGG_ERR_INVALID_ARG;
  }
  if (!out->keys || !is_device_ptr(out->keys)) return AGG_ERR_INVALID_ARG;
  if ((ops & AGG_COUNT) && !is_device_ptr(out->count)) return AGG_ERR_INVALID_ARG;
  if ((ops & AGG_SUM) && !is_device_ptr(out->sum)) return AGG_ERR_INVALID_ARG;
  if ((ops & AGG_MIN) && !is_device_ptr(out->min)) return AGG_ERR_INVALID_ARG;
  if ((ops & AGG_MAX) && !is_device_ptr(out->max)) return AGG_ERR_INVALID_ARG;
  if (uses_d_n_groups && out->d_n_groups && !is_device_ptr(out->d_n_groups)) return AGG_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_keys) & 7) ||
      (d_vals && (reinterpret_cast<uintptr_t>(d_vals) & (value_type == AGG_I64 ? 7 : 3))))
    return AGG_ERR_INVALID_ARG;
  return AGG_OK;
}

void free_staging(agg_handle* h) {
  for (int a = 0; a < 2; ++a) {
    if (h->stg_mem[a]) {
      if (h->stg_host) cudaFreeHost(h->stg_mem[a]);
      else cudaFree(h->stg_mem[a]);
    }
    h->stg_mem[a] = nullptr;
    h->stg[a] = nullptr;
    h->dir_part[a] = h->dir_count[a] = h->list[a] = nullptr;
  }
  h->max_chunks = 0;
  h->reserved_rows = 0;
  h->reserved_fan = 0;
  h->staging_bytes = 0;
  h->stg_host = false;
}

agg_status reserve_staging(agg_handle* h, uint64_t rows, uint32_t fan) {
  if (h->stg_mem[0] && rows <= h->reserved_rows && fan <= h->reserved_fan) return AGG_OK;
  if (rows < h->reserved_rows) rows = h->reserved_rows;
  if (fan < h->reserved_fan) fan = h->reserved_fan;
  free_staging(h);
  const uint64_t chunks = (rows + CH - 1) / CH + (uint64_t)h->ki.blocks * fan + 8;
  const uint64_t data = align_up(chunks * CH * REC_BYTES, 256);
  const uint64_t meta = align_up(chunks * 4, 256);
  const uint64_t per_area = data + 3 * meta;
  // device memory, or pinned host memory (mapped into the device's address
  // space) for the host tier, or when device memory cannot be had
  const uint32_t tier = h->tune.staging_tier;
  bool host = tier == 2;
  for (int attempt = 0; attempt < 2; ++attempt) {
    bool ok = true;
    for (int a = 0; a < 2 && ok; ++a) {
      void* m = nullptr;
      ok = (host ? cudaHostAlloc(&m, per_area, cudaHostAllocMapped | cudaHostAllocPortable)
                 : cudaMalloc(&m, per_area)) == cudaSuccess;
      if (ok) {
        h->stg_mem[a] = m;
        h->stg_host = host;
      }
    }
    if (ok) break;
    cudaGetLastError();
    free_staging(h);
    if (host || tier == 1) return AGG_ERR_OOM;
    host = true;  // the host tier
  }
  for (int a = 0; a < 2; ++a) {
    void* m = h->stg_mem[a];
    if (host) {
      void* dp = nullptr;
      if (cudaHostGetDevicePointer(&dp, m, 0) != cudaSuccess) {
        cudaGetLastError();
        free_staging(h);
        return AGG_ERR_CUDA;
      }
      m = dp;
    }
    uint8_t* b = static_cast<uint8_t*>(m);
    h->stg[a] = b;
    h->dir_part[a] = reinterpret_cast<uint32_t*>(b + data);
    h->dir_count[a] = reinterpret_cast<uint32_t*>(b + data + meta);
    h->list[a] = reinterpret_cast<uint32_t*>(b + data + 2 * meta);
  }
  h->max_chunks = chunks;
  h->reserved_rows = rows;
  h->reserved_fan = fan;
  h->staging_bytes = 2 * per_area;
  return AGG_OK;
}

agg_status reinit_working(agg_handle* h, cudaStream_t s) {
  if (cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) return AGG_ERR_CUDA;
  const unsigned long long none = ~0ull;
  if (cudaMemcpyAsync(&h->ctrl->rows_at_full, &none, 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return AGG_ERR_CUDA;
  if (hash_init_table(h->ent, h->tags, (uint32_t)h->slots, h->ent_kind, s) != cudaSuccess) return AGG_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return AGG_ERR_CUDA;
  h->dirty_lo = h->slots;
  h->table_dirty = false;
  return AGG_OK;
}

agg_status status_from_bits(unsigned long long bits) {
  const agg_status order[] = {AGG_ERR_TIMEOUT, AGG_ERR_INTERNAL, AGG_ERR_STAGING_EXHAUSTED, AGG_ERR_OUTPUT_CAPACITY};
  for (agg_status s : order)
    if (bits & (1ull << (int)s)) return s;
  return bits ? AGG_ERR_INTERNAL : AGG_OK;
}

agg_status hash_enqueue(agg_handle* h, const int64_t* d_keys, const void* d_vals, uint64_t n, const agg_output* out,
                        cudaStream_t s, bool host_input);
const void* device_view(const void* p, int device);

}  // namespace

extern "C" {

const char* agg_strerror(agg_status s) {
  switch (s) {
    case AGG_OK: return "ok";
    case AGG_ERR_INVALID_ARG: return "invalid argument";
    case AGG_ERR_BUDGET_TOO_SMALL: return "memory budget too small";
    case AGG_ERR_OOM: return "device memory allocation failed";
    case AGG_ERR_OUTPUT_CAPACITY: return "output capacity too small for the number of groups";
    case AGG_ERR_STAGING_EXHAUSTED: return "spill exceeded the reserved staging area";
    case AGG_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    case AGG_ERR_CUDA: return "CUDA runtime error";
    case AGG_ERR_INTERNAL: return "internal error";
  }
  return "unknown status";
}

agg_status agg_plan(size_t budget, const agg_spec* spec, const agg_tuning* t, uint64_t n, agg_plan_info* out) {
  if (!valid_spec(spec) || !out || !valid_tuning(t)) return AGG_ERR_INVALID_ARG;
  if (budget < AGG_MIN_BUDGET) return AGG_ERR_BUDGET_TOO_SMALL;
  const agg_tuning e = effective(t);
  const uint32_t es = entry_bytes(pick_ent(spec));
  Layout L;
  if (!layout_for(budget, es, &L)) return AGG_ERR_BUDGET_TOO_SMALL;
  out->entry_bytes = es;
  out->table_slots = L.slots;
  out->table_capacity = (uint64_t)(e.max_load_factor * (double)L.slots);
  out->fan_out = plan_fan(spec, e, n, budget, es);
  out->active_slots = active_slots(spec->expected_groups ? spec->expected_groups : (n ? n : 1),
                                   e.max_load_factor, L.slots, level0_cap(e));
  out->working_bytes = L.total;
  const uint64_t chunks = (n + CH - 1) / CH + 152ull * 2 * out->fan_out + 8;
  out->staging_bytes = 2 * (chunks * CH * REC_BYTES + 3 * chunks * 4);
  out->in_budget_path = 0;
  out->partitions = 0;
  const PathCosts pc = path_costs(spec, e, n, budget, es, L.slots);
  out->hash_bytes = pc.hash_bytes;
  out->sort_bytes = pc.sort_bytes;
  out->hash_seconds = pc.hash_s;
  out->sort_seconds = pc.sort_s;
  out->chosen_path = spec->path == AGG_PATH_AUTO ? (uint64_t)pc.choice : (uint64_t)spec->path;
  if (spec->path != AGG_PATH_SORT && out->chosen_path == AGG_PATH_HASH && e.in_budget != 2) {
    PartPlan pp;
    if (e.smem_entries != 1 && hash_part_plan(n, L.slots, es, e.smem_entries > 1 ? e.smem_entries : DEFAULT_NS, &pp)) {
      out->in_budget_path = 1;
      out->partitions = 1ull << pp.plog;
      out->active_slots = pp.s_ovf;
    } else if (const uint32_t sf = hash_fast_slots(n, L.slots)) {
      out->in_budget_path = 2;
      out->active_slots = sf;
    }
    if (out->in_budget_path) out->staging_bytes = 0;
  }
  return AGG_OK;
}

agg_status agg_create(size_t budget, const agg_spec* spec, agg_handle** out) {
  if (!out || !valid_spec(spec)) return AGG_ERR_INVALID_ARG;
  *out = nullptr;
  if (budget < AGG_MIN_BUDGET) return AGG_ERR_BUDGET_TOO_SMALL;
  agg_handle* h = new (std::nothrow) agg_handle();
  if (!h) return AGG_ERR_OOM;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return AGG_ERR_CUDA;
  }
  h->budget = budget;
  h->spec = *spec;
  h->tune = effective(nullptr);
  h->ent_kind = pick_ent(spec);
  h->es = entry_bytes(h->ent_kind);
  Layout L;
  if (!layout_for(budget, h->es, &L)) {
    delete h;
    return AGG_ERR_BUDGET_TOO_SMALL;
  }
  if (spec->path == AGG_PATH_SORT) {
    h->last_path = AGG_PATH_SORT;
    // sort path: the control block plus the sort's double buffers fill the budget
    const uint64_t cb = align_up(sizeof(Ctrl), 256);
    if (cudaMalloc(&h->work, cb) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return AGG_ERR_OOM;
    }
    h->ctrl = static_cast<Ctrl*>(h->work);
    if (cudaMallocHost(&h->ng_host, 64) != cudaSuccess || cudaMemset(h->ctrl, 0, sizeof(Ctrl)) != cudaSuccess) {
      cudaGetLastError();
      agg_destroy(h);
      return AGG_ERR_CUDA;
    }
    agg_status st = sort_reserve(h->sort, 0, budget - cb, *spec);
    if (st != AGG_OK) {
      agg_destroy(h);
      return st;
    }
    h->working_bytes = cb + h->sort.work_bytes;
    *out = h;
    return AGG_OK;
  }
  h->slots = L.slots;
  h->working_bytes = L.total;
  if (cudaMalloc(&h->work, L.total) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return AGG_ERR_OOM;
  }
  uint8_t* b = static_cast<uint8_t*>(h->work);
  h->ctrl = reinterpret_cast<Ctrl*>(b);
  h->tags = reinterpret_cast<uint32_t*>(b + L.tags_off);
  h->ent = b + L.ent_off;
  if (cudaMallocHost(&h->ng_host, 64) != cudaSuccess) {
    cudaGetLastError();
    agg_destroy(h);
    return AGG_ERR_OOM;
  }
  if (hash_kernel_info(h->ent_kind, spec->value_type, h->tune.smem_entries > 1 ? h->tune.smem_entries : DEFAULT_NS,
                       h->device, &h->ki) != cudaSuccess) {
    cudaGetLastError();
    agg_destroy(h);
    return AGG_ERR_CUDA;
  }
  agg_status st = reinit_working(h, nullptr);
  if (st != AGG_OK) {
    agg_destroy(h);
    return st;
  }
  if (spec->path == AGG_PATH_AUTO) {
    // the sort path of an AUTO handle works in the same memory, after the control block
    const uint64_t cb = align_up(sizeof(Ctrl), 256);
    sort_attach(h->sort, b + cb, L.total - cb);
  }
  *out = h;
  return AGG_OK;
}

agg_status agg_set_tuning(agg_handle* h, const agg_tuning* t) {
  if (!h || !valid_tuning(t)) return AGG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  const agg_tuning e = effective(t);
  if (h->spec.path == AGG_PATH_SORT) {
    h->tune = e;
    return AGG_OK;
  }
  KernelInfo ki;
  if (hash_kernel_info(h->ent_kind, h->spec.value_type, e.smem_entries > 1 ? e.smem_entries : DEFAULT_NS, h->device,
                       &ki) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  if (h->stg_mem[0] && e.staging_tier != 0 && (e.staging_tier == 2) != h->stg_host) {
    // another staging tier: reserved again on the next run
    cudaDeviceSynchronize();
    free_staging(h);
  }
  if (ki.blocks > h->ki.blocks && h->stg_mem[0]) {
    // more blocks means more open chunks: re-reserve on the next run
    const uint64_t rows = h->reserved_rows;
    const uint32_t fan = h->reserved_fan;
    cudaDeviceSynchronize();
    free_staging(h);
    h->ki = ki;
    h->tune = e;
    return reserve_staging(h, rows, fan);
  }
  h->ki = ki;
  h->tune = e;
  return AGG_OK;
}

agg_status agg_reserve(agg_handle* h, uint64_t max_rows) {
  if (!h) return AGG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  const uint32_t fan = plan_fan(&h->spec, h->tune, max_rows, h->budget, h->es);
  if (h->spec.path == AGG_PATH_SORT) {
    return sort_reserve(h->sort, max_rows, h->budget - align_up(sizeof(Ctrl), 256), h->spec);
  }
  return reserve_staging(h, max_rows, fan);
}

agg_status agg_run(agg_handle* h, const int64_t* d_keys, const void* d_vals, uint64_t n, const agg_output* out,
                   void* stream) {
  if (!h || !out) return AGG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const agg_status io = check_device_io(h->spec.ops, h->spec.value_type, d_keys, d_vals, n, out, true);
  if (io != AGG_OK) return io;

  int path = h->spec.path;
  if (path == AGG_PATH_AUTO) path = path_costs(&h->spec, h->tune, n, h->budget, h->es, h->slots).choice;
  if (path == AGG_PATH_SORT) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      return AGG_ERR_INVALID_ARG;  // the sort path plans on the host between kernels
    cudaGetLastError();
    agg_status st = sort_run(h->sort, h->budget - align_up(sizeof(Ctrl), 256), h->spec, h->ctrl, d_keys, d_vals, n,
                             out, s);
    h->last_stream = s;
    h->ran = true;
    h->last_path = AGG_PATH_SORT;
    if (h->spec.path == AGG_PATH_AUTO) h->table_dirty = true;
    return st;
  }
  if (h->table_dirty) {  // the sort path used the table's memory: clear it first
    if (hash_init_table(h->ent, h->tags, (uint32_t)h->slots, h->ent_kind, s) != cudaSuccess) {
      cudaGetLastError();
      return AGG_ERR_CUDA;
    }
    h->launches += 1;
    h->table_dirty = false;
    h->dirty_lo = h->slots;
  }
  h->last_path = AGG_PATH_HASH;
  return hash_enqueue(h, d_keys, d_vals, n, out, s, false);
}

}  // extern "C"

namespace {

// Enqueues the hash-path kernel.  Pointers are checked by the caller; they are
// device memory, or host memory the device can address when host_input is set
// (the kernel then streams the input over the host link and does not stage
// input tiles in L2 with bulk prefetches).
agg_status hash_enqueue(agg_handle* h, const int64_t* d_keys, const void* d_vals, uint64_t n, const agg_output* out,
                        cudaStream_t s, bool host_input) {
  const uint32_t fan = plan_fan(&h->spec, h->tune, n, h->budget, h->es);
  const uint32_t ns = h->tune.smem_entries > 1 ? h->tune.smem_entries : DEFAULT_NS;
  PartPlan pp;
  const bool in_budget = h->tune.in_budget != 2;
  const bool part = in_budget && h->tune.smem_entries != 1 && hash_part_plan(n, h->slots, h->es, ns, &pp);
  const uint32_t s_fast = part || !in_budget ? 0u : hash_fast_slots(n, h->slots);
  if (!part && !s_fast && (!h->stg_mem[0] || n > h->reserved_rows || fan > h->reserved_fan)) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      return AGG_ERR_INVALID_ARG;  // staging must be reserved before capture
    cudaGetLastError();
    agg_status st = reserve_staging(h, n, fan);
    if (st != AGG_OK) return st;
  }

  HashParams p{};
  p.keys = d_keys;
  p.vals = d_vals;
  p.n = n;
  p.has_vals = d_vals != nullptr;
  p.vec_ok = ((reinterpret_cast<uintptr_t>(d_keys) & 15) == 0) &&
             (!d_vals || (reinterpret_cast<uintptr_t>(d_vals) & (h->spec.value_type == AGG_I64 ? 15 : 7)) == 0);
  p.o_keys = out->keys;
  p.o_count = (h->spec.ops & AGG_COUNT) ? out->count : nullptr;
  p.o_sum = (h->spec.ops & AGG_SUM) ? out->sum : nullptr;
  p.o_min = (h->spec.ops & AGG_MIN) ? out->min : nullptr;
  p.o_max = (h->spec.ops & AGG_MAX) ? out->max : nullptr;
  p.o_cap = out->capacity;
  p.o_ngroups = out->d_n_groups;
  p.ctrl = h->ctrl;
  p.ent = h->ent;
  p.tags = h->tags;
  p.slots = (uint32_t)h->slots;
  for (int a = 0; a < 2; ++a) {
    p.stg[a] = h->stg[a];
    p.dir_part[a] = h->dir_part[a];
    p.dir_count[a] = h->dir_count[a];
    p.list[a] = h->list[a];
    p.max_chunks[a] = h->max_chunks;
  }
  p.seed = h->spec.seed;
  p.ops = h->spec.ops;
  p.fan_log2 = log2u(fan);
  p.lf = h->tune.max_load_factor;
  p.s_act0 = active_slots(h->spec.expected_groups ? h->spec.expected_groups : (n ? n : 1), p.lf, h->slots,
                          level0_cap(h->tune));
  p.ns = h->tune.smem_entries > 1 ? h->tune.smem_entries : DEFAULT_NS;
  p.cache = h->tune.smem_entries != 1;
  p.dedup = h->tune.warp_dedup == 1 ? 1 : 0;
  p.no_prefetch = host_input ? 1 : 0;
  p.stg_host = h->stg_host ? 1 : 0;
  hash_fallback_plan(fan, h->tune.max_levels, (uint32_t)h->ki.blocks, h->slots, h->es, p.ns, h->stg_mem[0] != nullptr,
                     &p);
  // the sorted-input path combines block boundaries with atomics on the output
  // rows: device outputs only
  p.sorted_probe = !host_input && h->tune.sorted_input != 2 && h->ki.blocks <= MAX_GRID ? 1 : 0;
  p.timeout_ns = h->tune.wait_limit_us ? 1000ull * h->tune.wait_limit_us : TIMEOUT_NS;
  // entries this run needs clear: the overflow table, the fast table, or all
  const uint64_t need_clear = part ? pp.s_ovf + 1ull : s_fast ? (uint64_t)s_fast : h->slots;
  if (h->dirty_lo < h->slots && need_clear > h->dirty_lo) {
    if (hash_reset_entries(h->ent + h->dirty_lo * h->es, h->slots - h->dirty_lo, h->ent_kind, s) != cudaSuccess) {
      cudaGetLastError();
      return AGG_ERR_CUDA;
    }
    h->launches += 1;
    h->dirty_lo = h->slots;
  }
  if (part) {
    // a small input: partitioned into shared-memory tables, no global atomics
    p.s_act0 = pp.s_ovf;
    if (hash_part_launch(h->ent_kind, h->spec.value_type, p, pp, h->es, h->ki.smem, s) != cudaSuccess) {
      cudaGetLastError();
      return AGG_ERR_CUDA;
    }
    h->dirty_lo = std::min<uint64_t>(h->dirty_lo, pp.scratch_slot);
    h->launches += 2;
    h->last_stream = s;
    h->ran = true;
    return AGG_OK;
  }
  if (s_fast) {
    // every distinct key fits: one pass in place, no spill, no grid barrier
    p.s_act0 = s_fast;
    if (hash_fast_launch(h->ent_kind, h->spec.value_type, p, s_fast, h->ki.smem, s) != cudaSuccess) {
      cudaGetLastError();
      return AGG_ERR_CUDA;
    }
    h->launches += n > 0 ? 2 : 1;
    h->last_stream = s;
    h->ran = true;
    return AGG_OK;
  }
  if (hash_launch(h->ent_kind, h->spec.value_type, p, h->ki, s) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  h->launches += 1;
  h->last_stream = s;
  h->ran = true;
  return AGG_OK;
}

// The address through which the device reaches host buffer p: the device
// pointer of pinned (registered) memory, or p itself when the device accesses
// pageable memory coherently (a Grace host over NVLink-C2C).  nullptr when the
// device cannot reach p.
const void* device_view(const void* p, int device) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (a.type == cudaMemoryTypeHost) return a.devicePointer;
  int pageable = 0;
  if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return pageable ? p : nullptr;
}

}  // namespace

extern "C" {

agg_status agg_sync(agg_handle* h, uint64_t* n_groups_host) {
  if (!h) return AGG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  unsigned long long bits = 0, ng = 0;
  if (cudaMemcpy(&bits, &h->ctrl->status_bits, 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&ng, &h->ctrl->last_n_groups, 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  if (n_groups_host) *n_groups_host = ng;
  const agg_status st = status_from_bits(bits);
  if (bits) {
    if (bits & ~(1ull << (int)AGG_ERR_OUTPUT_CAPACITY)) {
      // an aborted or inconsistent run may leave barrier or round state behind:
      // rebuild the working memory
      cudaDeviceSynchronize();
      agg_status r = h->spec.path == AGG_PATH_SORT ? AGG_OK : reinit_working(h, nullptr);
      if (h->spec.path == AGG_PATH_SORT) cudaMemset(h->ctrl, 0, sizeof(Ctrl));
      if (r != AGG_OK) return r;
    } else {
      unsigned long long zero = 0;
      cudaMemcpy(&h->ctrl->status_bits, &zero, 8, cudaMemcpyHostToDevice);
    }
  }
  return st;
}

agg_status agg_get_stats(agg_handle* h, agg_stats* s) {
  if (!h || !s) return AGG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  Ctrl c;
  if (cudaMemcpy(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  std::memset(s, 0, sizeof(*s));
  s->n_rows = c.last_n_rows;
  s->n_groups = c.last_n_groups;
  s->levels = c.last_levels;
  s->rounds = c.last_rounds;
  uint64_t spilled = 0;
  for (int l = 0; l < AGG_MAX_LEVELS; ++l) {
    s->spill_records[l] = c.last_spill_records[l];
    s->resident_groups[l] = c.last_resident_groups[l];
    spilled += c.last_spill_records[l];
  }
  s->spill_bytes_written = spilled * REC_BYTES;
  s->spill_bytes_read = spilled * REC_BYTES;
  s->rows_at_full = c.last_rows_at_full == ~0ull ? 0 : c.last_rows_at_full;
  for (int i = 0; i < PHASES; ++i) s->phase_ns[i] = c.last_phase_ns[i];
  s->table_slots = h->slots;
  s->table_capacity = (uint64_t)(h->tune.max_load_factor * (double)h->slots);
  s->table_bytes = h->working_bytes;
  s->budget_bytes = h->budget;
  s->staging_bytes = h->staging_bytes + sort_staging_bytes(h->sort);
  s->fan_out = plan_fan(&h->spec, h->tune, c.last_n_rows, h->budget, h->es);
  s->status_bits = c.status_bits;
  s->kernel_launches = h->launches + sort_launches(h->sort);
  s->sorted_input = c.last_sorted;
  s->fallback_records = c.last_fallback_records;
  s->fallback_level = c.last_fallback_level;
  s->staging_in_host = h->stg_host ? 1 : 0;
  s->path = (uint64_t)h->last_path;
  if (h->last_path == AGG_PATH_SORT) sort_fill_stats(h->sort, s);
  return AGG_OK;
}

agg_status agg_run_host(agg_handle* h, const int64_t* h_keys, const void* h_vals, uint64_t n, const agg_output* h_out,
                        uint64_t* n_groups, void* stream) {
  if (!h || !h_out || !h_out->keys || (n > 0 && !h_keys)) return AGG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t vb = h->spec.value_type == AGG_I64 ? 8 : 4;
  const uint64_t rows = n ? n : 1;
  const bool need_vals = (h->spec.ops & ~(uint32_t)AGG_COUNT) != 0;
  if (n > 0 && need_vals && !h_vals) return AGG_ERR_INVALID_ARG;

  // Direct mode (hash path): when the device can address every host buffer,
  // the kernel streams the input from host memory and writes the result rows
  // into the host arrays over the host link, overlapping both transfers with
  // its own work instead of copying before and after it.
  if (h->spec.path == AGG_PATH_HASH && n > 0) {
    const void* dk = device_view(h_keys, h->device);
    const void* dv = h_vals ? device_view(h_vals, h->device) : nullptr;
    agg_output dout{};
    dout.keys = static_cast<int64_t*>(const_cast<void*>(device_view(h_out->keys, h->device)));
    const uint32_t ops = h->spec.ops;
    dout.count = (ops & AGG_COUNT) && h_out->count
                     ? static_cast<uint64_t*>(const_cast<void*>(device_view(h_out->count, h->device)))
                     : nullptr;
    dout.sum = (ops & AGG_SUM) && h_out->sum ? static_cast<int64_t*>(const_cast<void*>(device_view(h_out->sum, h->device)))
                                             : nullptr;
    dout.min = (ops & AGG_MIN) && h_out->min ? static_cast<int64_t*>(const_cast<void*>(device_view(h_out->min, h->device)))
                                             : nullptr;
    dout.max = (ops & AGG_MAX) && h_out->max ? static_cast<int64_t*>(const_cast<void*>(device_view(h_out->max, h->device)))
                                             : nullptr;
    const bool direct = dk && (!h_vals || dv) && dout.keys && (!(ops & AGG_COUNT) || !h_out->count || dout.count) &&
                        (!(ops & AGG_SUM) || !h_out->sum || dout.sum) && (!(ops & AGG_MIN) || !h_out->min || dout.min) &&
                        (!(ops & AGG_MAX) || !h_out->max || dout.max) &&
                        (reinterpret_cast<uintptr_t>(dk) & 7) == 0 &&
                        (!dv || (reinterpret_cast<uintptr_t>(dv) & (vb - 1)) == 0);
    if (direct) {
      if (!h->out_buf) {
        if (cudaMalloc(&h->out_buf, 64) != cudaSuccess) {
          cudaGetLastError();
          return AGG_ERR_OOM;
        }
      }
      dout.capacity = h_out->capacity;
      dout.d_n_groups = static_cast<uint64_t*>(h->out_buf) + (h->out_cap ? h->out_cap * 5 : 0);
      agg_status st = hash_enqueue(h, static_cast<const int64_t*>(dk), dv, n, &dout, s, true);
      if (st != AGG_OK) return st;
      if (cudaMemcpyAsync(h->ng_host, dout.d_n_groups, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return AGG_ERR_CUDA;
      uint64_t ng = 0;
      st = agg_sync(h, &ng);
      ng = h->ng_host[0];
      if (n_groups) *n_groups = ng;
      if (st != AGG_OK) return st;
      return ng > h_out->capacity ? AGG_ERR_OUTPUT_CAPACITY : AGG_OK;
    }
  }
  if (rows > h->in_cap) {
    if (h->in_buf) cudaFree(h->in_buf);
    h->in_buf = nullptr;
    h->in_cap = 0;
    if (cudaMalloc(&h->in_buf, rows * (8 + 8)) != cudaSuccess) {
      cudaGetLastError();
      return AGG_ERR_OOM;
    }
    h->in_cap = rows;
  }
  if (rows > h->out_cap) {
    if (h->out_buf) cudaFree(h->out_buf);
    h->out_buf = nullptr;
    h->out_cap = 0;
    if (cudaMalloc(&h->out_buf, rows * 40 + 64) != cudaSuccess) {
      cudaGetLastError();
      return AGG_ERR_OOM;
    }
    h->out_cap = rows;
  }
  int64_t* dk = static_cast<int64_t*>(h->in_buf);
  void* dv = h_vals ? static_cast<void*>(static_cast<uint8_t*>(h->in_buf) + rows * 8) : nullptr;
  uint8_t* ob = static_cast<uint8_t*>(h->out_buf);
  agg_output dout{};
  dout.keys = reinterpret_cast<int64_t*>(ob);
  dout.count = reinterpret_cast<uint64_t*>(ob + rows * 8);
  dout.sum = reinterpret_cast<int64_t*>(ob + rows * 16);
  dout.min = reinterpret_cast<int64_t*>(ob + rows * 24);
  dout.max = reinterpret_cast<int64_t*>(ob + rows * 32);
  dout.capacity = rows;
  dout.d_n_groups = reinterpret_cast<uint64_t*>(ob + rows * 40);
  if (n > 0) {
    if (cudaMemcpyAsync(dk, h_keys, n * 8, cudaMemcpyDefault, s) != cudaSuccess) return AGG_ERR_CUDA;
    if (dv && cudaMemcpyAsync(dv, h_vals, n * vb, cudaMemcpyDefault, s) != cudaSuccess) return AGG_ERR_CUDA;
  }
  agg_status st = agg_run(h, dk, dv, n, &dout, stream);
  if (st != AGG_OK) return st;
  if (cudaMemcpyAsync(h->ng_host, dout.d_n_groups, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return AGG_ERR_CUDA;
  uint64_t ng = 0;
  st = agg_sync(h, &ng);
  if (st != AGG_OK) return st;
  ng = h->ng_host[0];
  if (n_groups) *n_groups = ng;
  if (ng > h_out->capacity) return AGG_ERR_OUTPUT_CAPACITY;
  if (ng > 0) {
    struct {
      void* dst;
      const void* src;
      bool want;
    } cp[5] = {{h_out->keys, dout.keys, true},
               {h_out->count, dout.count, (h->spec.ops & AGG_COUNT) != 0},
               {h_out->sum, dout.sum, (h->spec.ops & AGG_SUM) != 0},
               {h_out->min, dout.min, (h->spec.ops & AGG_MIN) != 0},
               {h_out->max, dout.max, (h->spec.ops & AGG_MAX) != 0}};
    for (auto& c : cp)
      if (c.want && c.dst && cudaMemcpyAsync(c.dst, c.src, ng * 8, cudaMemcpyDefault, s) != cudaSuccess)
        return AGG_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return AGG_ERR_CUDA;
  return AGG_OK;
}

agg_status agg_destroy(agg_handle* h) {
  if (!h) return AGG_OK;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  cudaGetLastError();
  free_staging(h);
  sort_free(h->sort);
  if (h->work) cudaFree(h->work);
  if (h->in_buf) cudaFree(h->in_buf);
  if (h->out_buf) cudaFree(h->out_buf);
  if (h->ng_host) cudaFreeHost(h->ng_host);
  delete h;
  return AGG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batched form

struct agg_batch {
  int device = 0;
  agg_spec spec{};
  int ent_kind = 0;
  uint32_t es = 32;
  uint32_t count = 0;
  uint32_t team_blocks = 4, nteams = 0;
  KernelInfo ki{};
  void* work = nullptr;     // all teams' working memory
  void* staging = nullptr;  // all teams' staging areas
  HashParams* d_items = nullptr;
  uint32_t* d_team_off = nullptr;
  uint32_t* d_team_items = nullptr;
  unsigned long long* d_ngroups = nullptr;
  std::vector<Ctrl*> ctrl;
  std::vector<uint8_t*> team_ent;
  std::vector<uint32_t*> team_tags;
  std::vector<uint32_t> team_slots;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = true;
  cudaStream_t last_stream = nullptr;
};

namespace {

agg_status batch_init_teams(agg_batch* b) {
  for (uint32_t t = 0; t < b->nteams; ++t) {
    if (cudaMemset(b->ctrl[t], 0, sizeof(Ctrl)) != cudaSuccess ||
        hash_init_table(b->team_ent[t], b->team_tags[t], b->team_slots[t], b->ent_kind, nullptr) != cudaSuccess)
      return AGG_ERR_CUDA;
  }
  return cudaDeviceSynchronize() == cudaSuccess ? AGG_OK : AGG_ERR_CUDA;
}

agg_status batch_launch(agg_batch* b, cudaStream_t s) {
  return hash_batch_launch(b->ent_kind, b->spec.value_type, b->d_items, b->d_team_off, b->d_team_items,
                           b->team_blocks, b->nteams, b->ki.smem, s) == cudaSuccess
             ? AGG_OK
             : AGG_ERR_CUDA;
}

}  // namespace

extern "C" {

agg_status agg_batch_create(const agg_spec* spec, const agg_batch_item* items, uint32_t count,
                            const agg_batch_tuning* t, agg_batch** out) {
  if (!out || !valid_spec(spec) || spec->path != AGG_PATH_HASH || (count > 0 && !items)) return AGG_ERR_INVALID_ARG;
  *out = nullptr;
  if (t && ((t->team_blocks & (t->team_blocks - 1)) || (t->smem_entries && (t->smem_entries < 512 ||
      t->smem_entries > 4096 || (t->smem_entries & (t->smem_entries - 1)))) || t->max_load_factor < 0 ||
      t->max_load_factor > 0.95 || (t->fan_out && (t->fan_out < 16 || t->fan_out > 256 ||
      (t->fan_out & (t->fan_out - 1)))) || t->use_graph > 2))
    return AGG_ERR_INVALID_ARG;
  agg_batch* b = new (std::nothrow) agg_batch();
  if (!b) return AGG_ERR_OOM;
  auto fail = [&](agg_status st) {
    agg_batch_destroy(b);
    return st;
  };
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return AGG_ERR_CUDA;
  }
  b->spec = *spec;
  b->count = count;
  b->ent_kind = pick_ent(spec);
  b->es = entry_bytes(b->ent_kind);
  b->use_graph = !(t && t->use_graph == 2);
  agg_tuning tune = effective(nullptr);
  if (t && t->smem_entries) tune.smem_entries = t->smem_entries;
  if (t && t->max_load_factor > 0) tune.max_load_factor = t->max_load_factor;
  if (t && t->fan_out) tune.fan_out = t->fan_out;
  if (hash_batch_kernel_info(b->ent_kind, spec->value_type, tune.smem_entries, b->device, &b->ki) != cudaSuccess) {
    cudaGetLastError();
    return fail(AGG_ERR_CUDA);
  }
  b->team_blocks = (t && t->team_blocks) ? t->team_blocks : 4;
  while (b->team_blocks > 1 && (uint32_t)b->ki.blocks < b->team_blocks) b->team_blocks >>= 1;
  b->nteams = (uint32_t)b->ki.blocks / b->team_blocks;

  // per-instance plan
  struct Plan {
    uint64_t slots, fan, s_act0;
    bool may_spill;
  };
  std::vector<Plan> plan(count);
  for (uint32_t i = 0; i < count; ++i) {
    const agg_status io =
        check_device_io(spec->ops, spec->value_type, items[i].d_keys, items[i].d_vals, items[i].n, &items[i].out, false);
    if (io != AGG_OK) return fail(io);
    Layout L;
    if (!layout_for(items[i].budget, b->es, &L)) return fail(AGG_ERR_BUDGET_TOO_SMALL);
    agg_spec si = *spec;
    si.expected_groups = items[i].expected_groups;
    const uint64_t est = si.expected_groups ? si.expected_groups : (items[i].n ? items[i].n : 1);
    uint64_t need = (uint64_t)((double)(items[i].n ? items[i].n : 1) / tune.max_load_factor) + BUCKET;
    need = std::max<uint64_t>((need + BUCKET - 1) / BUCKET * BUCKET, 2 * MIN_SLOTS);
    plan[i].slots = std::min<uint64_t>(L.slots, need);  // never more than the input can use
    plan[i].s_act0 = active_slots(est, tune.max_load_factor, plan[i].slots, level0_cap(tune));
    plan[i].fan = plan_fan(&si, tune, items[i].n, items[i].budget, b->es);
    plan[i].may_spill = items[i].n > (uint64_t)(0.5 * (double)plan[i].slots);
  }
  // teams: longest first onto the least loaded team (each instance also costs a fixed overhead)
  std::vector<uint32_t> order(count);
  for (uint32_t i = 0; i < count; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t c) { return items[a].n > items[c].n; });
  using Load = std::pair<double, uint32_t>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (uint32_t tm = 0; tm < b->nteams; ++tm) heap.push({0.0, tm});
  std::vector<std::vector<uint32_t>> lists(b->nteams);
  for (uint32_t i : order) {
    Load l = heap.top();
    heap.pop();
    lists[l.second].push_back(i);
    l.first += (double)items[i].n + 20000.0;
    heap.push(l);
  }
  // memory: per team, room for its largest table and its largest spilling input
  std::vector<uint64_t> slots_t(b->nteams, 2 * MIN_SLOTS), rows_t(b->nteams, 0), fan_t(b->nteams, 16);
  for (uint32_t tm = 0; tm < b->nteams; ++tm)
    for (uint32_t i : lists[tm]) {
      slots_t[tm] = std::max<uint64_t>(slots_t[tm], plan[i].slots);
      if (plan[i].may_spill) rows_t[tm] = std::max<uint64_t>(rows_t[tm], items[i].n);
      fan_t[tm] = std::max<uint64_t>(fan_t[tm], plan[i].fan);
    }
  const uint64_t ctrl_bytes = align_up(sizeof(Ctrl), 256);
  std::vector<uint64_t> woff(b->nteams + 1, 0), soff(b->nteams + 1, 0), chunks_t(b->nteams, 0);
  for (uint32_t tm = 0; tm < b->nteams; ++tm) {
    const uint64_t tags = align_up(slots_t[tm] + BUCKET, 256);
    woff[tm + 1] = woff[tm] + align_up(ctrl_bytes + tags + (slots_t[tm] + 1) * b->es, 256);
    if (rows_t[tm]) chunks_t[tm] = (rows_t[tm] + CH - 1) / CH + (uint64_t)b->team_blocks * fan_t[tm] + 8;
    const uint64_t per_area = align_up(chunks_t[tm] * CH * REC_BYTES, 256) + 3 * align_up(chunks_t[tm] * 4, 256);
    soff[tm + 1] = soff[tm] + 2 * per_area;
  }
  if (cudaMalloc(&b->work, std::max<uint64_t>(woff[b->nteams], 256)) != cudaSuccess ||
      (soff[b->nteams] && cudaMalloc(&b->staging, soff[b->nteams]) != cudaSuccess) ||
      cudaMalloc(&b->d_ngroups, std::max<uint64_t>(count, 1) * 8) != cudaSuccess) {
    cudaGetLastError();
    return fail(AGG_ERR_OOM);
  }
  b->ctrl.resize(b->nteams);
  b->team_ent.resize(b->nteams);
  b->team_tags.resize(b->nteams);
  b->team_slots.resize(b->nteams);
  std::vector<HashParams> hp(count);
  for (uint32_t tm = 0; tm < b->nteams; ++tm) {
    uint8_t* base = static_cast<uint8_t*>(b->work) + woff[tm];
    const uint64_t tags = align_up(slots_t[tm] + BUCKET, 256);
    b->ctrl[tm] = reinterpret_cast<Ctrl*>(base);
    b->team_tags[tm] = reinterpret_cast<uint32_t*>(base + ctrl_bytes);
    b->team_ent[tm] = base + ctrl_bytes + tags;
    b->team_slots[tm] = (uint32_t)slots_t[tm];
    uint8_t* stg = b->staging ? static_cast<uint8_t*>(b->staging) + soff[tm] : nullptr;
    const uint64_t data = align_up(chunks_t[tm] * CH * REC_BYTES, 256), meta = align_up(chunks_t[tm] * 4, 256);
    for (uint32_t i : lists[tm]) {
      HashParams& p = hp[i];
      const agg_batch_item& it = items[i];
      p.keys = it.d_keys;
      p.vals = it.d_vals;
      p.n = it.n;
      p.has_vals = it.d_vals != nullptr;
      p.vec_ok = ((reinterpret_cast<uintptr_t>(it.d_keys) & 15) == 0) &&
                 (!it.d_vals || (reinterpret_cast<uintptr_t>(it.d_vals) & (spec->value_type == AGG_I64 ? 15 : 7)) == 0);
      p.o_keys = it.out.keys;
      p.o_count = (spec->ops & AGG_COUNT) ? it.out.count : nullptr;
      p.o_sum = (spec->ops & AGG_SUM) ? it.out.sum : nullptr;
      p.o_min = (spec->ops & AGG_MIN) ? it.out.min : nullptr;
      p.o_max = (spec->ops & AGG_MAX) ? it.out.max : nullptr;
      p.o_cap = it.out.capacity;
      p.o_ngroups = reinterpret_cast<uint64_t*>(b->d_ngroups + i);
      p.ctrl = b->ctrl[tm];
      p.ent = b->team_ent[tm];
      p.tags = b->team_tags[tm];
      p.slots = (uint32_t)plan[i].slots;
      for (int a = 0; a < 2; ++a) {
        uint8_t* area = stg ? stg + a * (data + 3 * meta) : nullptr;
        p.stg[a] = area;
        p.dir_part[a] = area ? reinterpret_cast<uint32_t*>(area + data) : nullptr;
        p.dir_count[a] = area ? reinterpret_cast<uint32_t*>(area + data + meta) : nullptr;
        p.list[a] = area ? reinterpret_cast<uint32_t*>(area + data + 2 * meta) : nullptr;
        p.max_chunks[a] = area ? chunks_t[tm] : 0;
      }
      p.seed = spec->seed + i;
      p.ops = spec->ops;
      p.fan_log2 = log2u((uint32_t)plan[i].fan);
      p.lf = tune.max_load_factor;
      p.s_act0 = (uint32_t)plan[i].s_act0;
      p.ns = tune.smem_entries;
      p.cache = 1;
      p.dedup = tune.warp_dedup == 1 ? 1 : 0;
      p.timeout_ns = TIMEOUT_NS;
      hash_fallback_plan((uint32_t)plan[i].fan, 0, b->team_blocks, plan[i].slots, b->es, p.ns, p.stg[0] != nullptr, &p);
    }
  }
  std::vector<uint32_t> toff(b->nteams + 1, 0), titems;
  titems.reserve(count);
  for (uint32_t tm = 0; tm < b->nteams; ++tm) {
    toff[tm + 1] = toff[tm] + (uint32_t)lists[tm].size();
    titems.insert(titems.end(), lists[tm].begin(), lists[tm].end());
  }
  if (cudaMalloc(&b->d_items, std::max<uint64_t>(count, 1) * sizeof(HashParams)) != cudaSuccess ||
      cudaMalloc(&b->d_team_off, (b->nteams + 1) * 4) != cudaSuccess ||
      cudaMalloc(&b->d_team_items, std::max<uint64_t>(count, 1) * 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(AGG_ERR_OOM);
  }
  if ((count && cudaMemcpy(b->d_items, hp.data(), count * sizeof(HashParams), cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(b->d_team_off, toff.data(), (b->nteams + 1) * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      (count && cudaMemcpy(b->d_team_items, titems.data(), count * 4, cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemset(b->d_ngroups, 0, std::max<uint64_t>(count, 1) * 8) != cudaSuccess) {
    cudaGetLastError();
    return fail(AGG_ERR_CUDA);
  }
  agg_status st = batch_init_teams(b);
  if (st != AGG_OK) return fail(st);
  *out = b;
  return AGG_OK;
}

agg_status agg_batch_run(agg_batch* b, void* stream) {
  if (!b) return AGG_ERR_INVALID_ARG;
  DeviceGuard g(b->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  b->last_stream = s;
  if (b->use_graph && !b->exec) {
    // capture the one launch of the batch kernel as a graph, once
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const agg_status ls = batch_launch(b, cs);
      ok = cudaStreamEndCapture(cs, &graph) == cudaSuccess && ls == AGG_OK && graph &&
           cudaGraphInstantiate(&b->exec, graph, 0) == cudaSuccess;
    }
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    if (!ok) {
      cudaGetLastError();
      b->exec = nullptr;
      b->use_graph = false;  // launch directly from now on
    }
  }
  if (b->exec) return cudaGraphLaunch(b->exec, s) == cudaSuccess ? AGG_OK : AGG_ERR_CUDA;
  return batch_launch(b, s);
}

agg_status agg_batch_sync(agg_batch* b, uint64_t* n_groups) {
  if (!b) return AGG_ERR_INVALID_ARG;
  DeviceGuard g(b->device);
  if (cudaStreamSynchronize(b->last_stream) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  unsigned long long bits = 0;
  for (uint32_t tm = 0; tm < b->nteams; ++tm) {
    unsigned long long x = 0;
    if (cudaMemcpy(&x, &b->ctrl[tm]->status_bits, 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return AGG_ERR_CUDA;
    }
    bits |= x;
  }
  if (n_groups && b->count &&
      cudaMemcpy(n_groups, b->d_ngroups, (size_t)b->count * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  if (bits) {
    const agg_status st = status_from_bits(bits);
    const agg_status r = batch_init_teams(b);  // clear every team's state for the next run
    return r != AGG_OK ? r : st;
  }
  return AGG_OK;
}

agg_status agg_batch_destroy(agg_batch* b) {
  if (!b) return AGG_OK;
  DeviceGuard g(b->device);
  cudaDeviceSynchronize();
  cudaGetLastError();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->work) cudaFree(b->work);
  if (b->staging) cudaFree(b->staging);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_team_off) cudaFree(b->d_team_off);
  if (b->d_team_items) cudaFree(b->d_team_items);
  if (b->d_ngroups) cudaFree(b->d_ngroups);
  delete b;
  return AGG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- served form

struct ServerQuery {
  agg_query q{};
  agg_query_info info{};
  uint64_t pool_off = 0, pool_len = 0;  // working memory (declared budget) in the pool
  uint64_t stg_off = 0, stg_len = 0;    // staging in the staging pool (0 when the query cannot spill)
  uint32_t team = 0;                    // thread blocks it holds while it runs
  int slot = -1;
};

// One pool of device memory carved into ranges (first fit, neighbours merged).
struct RangePool {
  uint8_t* base = nullptr;
  uint64_t bytes = 0, in_use = 0, peak = 0;
  std::map<uint64_t, uint64_t> free_list;  // offset -> length
};

struct agg_server {
  int device = 0;
  agg_spec spec{};
  int ent_kind = 0;
  uint32_t es = 32;
  agg_tuning tune{};
  KernelInfo ki{};  // launch shape of one block team (smem) and the whole-GPU block count
  void* mem = nullptr;  // one allocation: the working-memory pool, then the staging pool
  RangePool pool;       // declared budgets of admitted queries (Section 3.2)
  RangePool stage;      // their staging areas (outside the budgets, like the paper's disk)
  uint32_t blocks_in_use = 0, big_blocks_in_use = 0;
  uint32_t inject_fail_at = 0;  // test hook: the k-th launch (1-based) fails after its set-up was queued
  uint32_t sort_epoch = 0;      // look-back epochs of the sort runs (each run's memory is cleared first)
  uint32_t launches = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<int64_t> slot_ticket;  // -1 = free
  unsigned long long* pinned = nullptr;  // per slot: status bits, group count
  std::deque<uint64_t> waiting;
  std::unordered_map<uint64_t, ServerQuery> queries;
  uint64_t next_ticket = 1;
  uint64_t submitted = 0, completed = 0, running = 0, max_conc = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

bool pool_alloc(RangePool& p, uint64_t len, uint64_t* off) {
  len = align_up(len, 256);
  if (len == 0) {
    *off = 0;
    return true;
  }
  for (auto it = p.free_list.begin(); it != p.free_list.end(); ++it) {
    if (it->second < len) continue;
    *off = it->first;
    const uint64_t rest = it->second - len, roff = it->first + len;
    p.free_list.erase(it);
    if (rest) p.free_list[roff] = rest;
    p.in_use += len;
    p.peak = std::max(p.peak, p.in_use);
    return true;
  }
  return false;
}

void pool_free(RangePool& p, uint64_t off, uint64_t len) {
  len = align_up(len, 256);
  if (len == 0) return;
  p.in_use -= len;
  auto it = p.free_list.emplace(off, len).first;
  auto nx = std::next(it);
  if (nx != p.free_list.end() && it->first + it->second == nx->first) {  // merge with the next
    it->second += nx->second;
    p.free_list.erase(nx);
  }
  if (it != p.free_list.begin()) {  // merge with the previous
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      p.free_list.erase(it);
    }
  }
}

// Thread blocks a query would like: about 8k rows per block (four tiles), a
// power of two from 8 to the whole GPU.  A server that runs one query at a
// time gives each query the whole GPU.
uint32_t team_wanted(uint64_t n, uint32_t all_blocks, uint32_t max_active) {
  if (max_active == 1) return all_blocks;
  uint32_t b = 8;
  while (b < all_blocks && (uint64_t)b * 8192 < n) b <<= 1;
  return std::min(b, all_blocks);
}

// Queries that want more than SMALL_TEAM blocks are "big"; together they may
// hold at most all_blocks - all_blocks / SMALL_RESERVE_DIV blocks, so that
// the small queries (most arrivals) always find blocks free at once instead of
// waiting behind a long query.
constexpr uint32_t SMALL_TEAM = 32;
constexpr uint32_t SMALL_RESERVE_DIV = 4;

struct QueryPlan {
  Layout L;
  uint64_t slots = 0, chunks = 0, data = 0, meta = 0, stg_len = 0;
  uint32_t fan = 16, team = 0;
  bool may_spill = false;
  int in_budget = 0;      // 1 partitioned, 2 single table (ordinary launches, no team), 0 the spilling kernel
  PartPlan pp;
  uint32_t s_fast = 0;
  bool sort = false;      // the sort path in the query's working memory (one round: no host step)
};

// Table size, fan-out and staging of a query run by `team` blocks.
QueryPlan plan_query(const agg_server* s, const agg_query& q, uint32_t team) {
  QueryPlan P;
  layout_for(q.budget, s->es, &P.L);
  const uint64_t n = q.n;
  uint64_t need = (uint64_t)((double)(n ? n : 1) / s->tune.max_load_factor) + BUCKET;
  need = std::max<uint64_t>((need + BUCKET - 1) / BUCKET * BUCKET, 2 * MIN_SLOTS);
  P.slots = std::min<uint64_t>(P.L.slots, need);
  P.may_spill = n > (uint64_t)(0.5 * (double)P.slots);
  agg_spec si = s->spec;
  si.expected_groups = q.expected_groups;
  P.fan = plan_fan(&si, s->tune, n, q.budget, s->es);
  P.team = team;
  if (s->spec.path == AGG_PATH_AUTO &&
      path_costs(&si, s->tune, n, q.budget, s->es, P.L.slots).choice == AGG_PATH_SORT) {
    const uint64_t cb = align_up(sizeof(Ctrl), 256);
    if (n <= sort_rows_for(P.L.total - cb)) {  // one sort round: nothing for the host to plan
      P.sort = true;
      P.team = 0;
      P.may_spill = false;
      return P;
    }
  }
  // every group fits the table at once: the in-budget paths, no staging
  const uint32_t ns = s->tune.smem_entries;
  if (hash_part_plan(n, P.slots, s->es, ns, &P.pp)) {
    P.in_budget = 1;
  } else if ((P.s_fast = hash_fast_slots(n, P.slots)) != 0) {
    P.in_budget = 2;
  }
  if (P.in_budget) {
    P.team = 0;
    P.may_spill = false;
    return P;
  }
  if (P.may_spill) {
    P.chunks = (n + CH - 1) / CH + (uint64_t)team * P.fan + 8;
    P.data = align_up(P.chunks * CH * REC_BYTES, 256);
    P.meta = align_up(P.chunks * 4, 256);
    P.stg_len = 2 * (P.data + 3 * P.meta);
  }
  return P;
}

// Enqueues the set-up and the kernel of an admitted query on its slot's stream.
// On an error the caller must let the slot's stream drain before it frees the
// query's pool ranges (work queued before the error may still use them).
agg_status server_launch(agg_server* s, ServerQuery& sq, const QueryPlan& P, int slot) {
  cudaStream_t st = s->streams[slot];
  const agg_query& q = sq.q;
  uint8_t* base = s->pool.base + sq.pool_off;
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(base);
  uint32_t* tags = reinterpret_cast<uint32_t*>(base + P.L.tags_off);
  uint8_t* ent = base + P.L.ent_off;
  const uint64_t n = q.n;
  if (q.ready && cudaStreamWaitEvent(st, static_cast<cudaEvent_t>(q.ready), 0) != cudaSuccess) return AGG_ERR_CUDA;
  if (P.sort) {  // the sort path, in the query's working memory after its control block
    if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return AGG_ERR_CUDA;
    s->launches += 1;
    if (s->inject_fail_at && s->launches == s->inject_fail_at) return AGG_ERR_CUDA;  // host-injected failure
    const uint64_t cb = align_up(sizeof(Ctrl), 256);
    SortState ss{};
    sort_attach(ss, base + cb, P.L.total - cb);
    ss.epoch = s->sort_epoch;
    agg_output o = q.out;
    o.d_n_groups = nullptr;
    const agg_status r = sort_run(ss, P.L.total - cb, s->spec, ctrl, q.d_keys, q.d_vals, n, &o, st);
    s->sort_epoch = ss.epoch;
    if (r != AGG_OK) return r;
    if (cudaMemcpyAsync(s->pinned + 2 * slot, &ctrl->status_bits, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(s->pinned + 2 * slot + 1, &ctrl->last_n_groups, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(s->events[slot], st) != cudaSuccess)
      return AGG_ERR_CUDA;
    sq.info.team_blocks = 0;
    sq.info.path = AGG_PATH_SORT;
    return AGG_OK;
  }
  // the entries this run uses (and the side slot after them) start empty
  const uint32_t used = P.in_budget == 1 ? P.pp.s_ovf : P.in_budget == 2 ? P.s_fast : (uint32_t)P.slots;
  if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st) != cudaSuccess ||
      hash_init_table(ent, tags, used, s->ent_kind, st) != cudaSuccess)
    return AGG_ERR_CUDA;
  s->launches += 1;
  if (s->inject_fail_at && s->launches == s->inject_fail_at) return AGG_ERR_CUDA;  // host-injected failure
  HashParams p{};
  uint8_t* stg = P.stg_len ? s->stage.base + sq.stg_off : nullptr;
  for (int a = 0; a < 2; ++a) {
    uint8_t* area = stg ? stg + a * (P.data + 3 * P.meta) : nullptr;
    p.stg[a] = area;
    p.dir_part[a] = area ? reinterpret_cast<uint32_t*>(area + P.data) : nullptr;
    p.dir_count[a] = area ? reinterpret_cast<uint32_t*>(area + P.data + P.meta) : nullptr;
    p.list[a] = area ? reinterpret_cast<uint32_t*>(area + P.data + 2 * P.meta) : nullptr;
    p.max_chunks[a] = area ? P.chunks : 0;
  }
  p.keys = q.d_keys;
  p.vals = q.d_vals;
  p.n = n;
  p.has_vals = q.d_vals != nullptr;
  p.vec_ok = ((reinterpret_cast<uintptr_t>(q.d_keys) & 15) == 0) &&
             (!q.d_vals || (reinterpret_cast<uintptr_t>(q.d_vals) & (s->spec.value_type == AGG_I64 ? 15 : 7)) == 0);
  p.o_keys = q.out.keys;
  p.o_count = (s->spec.ops & AGG_COUNT) ? q.out.count : nullptr;
  p.o_sum = (s->spec.ops & AGG_SUM) ? q.out.sum : nullptr;
  p.o_min = (s->spec.ops & AGG_MIN) ? q.out.min : nullptr;
  p.o_max = (s->spec.ops & AGG_MAX) ? q.out.max : nullptr;
  p.o_cap = q.out.capacity;
  p.o_ngroups = nullptr;
  p.ctrl = ctrl;
  p.ent = ent;
  p.tags = tags;
  p.slots = used;  // the side slot follows the entries in use
  p.seed = s->spec.seed;
  p.ops = s->spec.ops;
  p.fan_log2 = log2u(P.fan);
  p.lf = s->tune.max_load_factor;
  p.s_act0 = active_slots(q.expected_groups ? q.expected_groups : (n ? n : 1), p.lf, P.slots,
                          level0_cap(s->tune));
  p.ns = s->tune.smem_entries;
  p.cache = 1;
  p.dedup = s->tune.warp_dedup == 1 ? 1 : 0;
  p.timeout_ns = TIMEOUT_NS;
  if (P.in_budget == 1) {
    // the scratch of the partitions lies above the overflow table and its side slot
    p.s_act0 = P.pp.s_ovf;
    if (hash_part_launch(s->ent_kind, s->spec.value_type, p, P.pp, s->es, s->ki.smem, st) != cudaSuccess)
      return AGG_ERR_CUDA;
  } else if (P.in_budget == 2) {
    p.s_act0 = P.s_fast;
    if (hash_fast_launch(s->ent_kind, s->spec.value_type, p, P.s_fast, s->ki.smem, st) != cudaSuccess)
      return AGG_ERR_CUDA;
  } else {
    hash_fallback_plan(P.fan, 0, P.team, P.slots, s->es, p.ns, p.stg[0] != nullptr, &p);
    KernelInfo ki = s->ki;
    ki.blocks = (int)P.team;
    if (hash_launch(s->ent_kind, s->spec.value_type, p, ki, st) != cudaSuccess) return AGG_ERR_CUDA;
  }
  if (cudaMemcpyAsync(s->pinned + 2 * slot, &ctrl->status_bits, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(s->pinned + 2 * slot + 1, &ctrl->last_n_groups, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaEventRecord(s->events[slot], st) != cudaSuccess)
    return AGG_ERR_CUDA;
  sq.info.team_blocks = P.team;
  sq.info.path = AGG_PATH_HASH;
  return AGG_OK;
}

void release_query(agg_server* s, ServerQuery& sq) {
  pool_free(s->pool, sq.pool_off, sq.pool_len);
  pool_free(s->stage, sq.stg_off, sq.stg_len);
  sq.pool_len = sq.stg_len = 0;
  s->blocks_in_use -= sq.team;
  if (sq.team > SMALL_TEAM) s->big_blocks_in_use -= sq.team;
  sq.team = 0;
}

}  // namespace

extern "C" {

agg_status agg_server_create(const agg_spec* spec, size_t pool_bytes, uint32_t max_active, agg_server** out) {
  if (!out || !valid_spec(spec) || spec->path == AGG_PATH_SORT || max_active == 0 || max_active > 4096 ||
      pool_bytes < AGG_MIN_BUDGET)
    return AGG_ERR_INVALID_ARG;
  *out = nullptr;
  agg_server* s = new (std::nothrow) agg_server();
  if (!s) return AGG_ERR_OOM;
  auto fail = [&](agg_status st) {
    agg_server_destroy(s);
    return st;
  };
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return AGG_ERR_CUDA;
  }
  s->spec = *spec;
  s->ent_kind = pick_ent(spec);
  s->es = entry_bytes(s->ent_kind);
  s->tune = effective(nullptr);
  if (const char* e = std::getenv("AGG_INJECT_LAUNCH_FAILURE")) s->inject_fail_at = (uint32_t)std::strtoul(e, nullptr, 10);
  if (hash_kernel_info(s->ent_kind, spec->value_type, s->tune.smem_entries, s->device, &s->ki) != cudaSuccess) {
    cudaGetLastError();
    return fail(AGG_ERR_CUDA);
  }
  const uint64_t pool = align_up(pool_bytes, 256);
  const uint64_t stage = align_up(std::max<uint64_t>(pool_bytes / 2, AGG_SERVER_MIN_STAGING), 256);
  if (cudaMalloc(&s->mem, pool + stage) != cudaSuccess) {
    cudaGetLastError();
    return fail(AGG_ERR_OOM);
  }
  s->pool.base = static_cast<uint8_t*>(s->mem);
  s->pool.bytes = pool_bytes;
  s->pool.free_list[0] = pool_bytes;
  s->stage.base = static_cast<uint8_t*>(s->mem) + pool;
  s->stage.bytes = stage;
  s->stage.free_list[0] = stage;
  if (cudaMallocHost(reinterpret_cast<void**>(&s->pinned), 16ull * max_active) != cudaSuccess) {
    cudaGetLastError();
    return fail(AGG_ERR_OOM);
  }
  s->streams.resize(max_active, nullptr);
  s->events.resize(max_active, nullptr);
  s->slot_ticket.assign(max_active, -1);
  for (uint32_t i = 0; i < max_active; ++i)
    if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(AGG_ERR_CUDA);
    }
  *out = s;
  return AGG_OK;
}

agg_status agg_server_submit(agg_server* s, const agg_query* q, uint64_t* ticket) {
  if (!s || !q || !ticket) return AGG_ERR_INVALID_ARG;
  Layout L;
  if (!layout_for(q->budget, s->es, &L)) return AGG_ERR_BUDGET_TOO_SMALL;
  if (L.total > s->pool.bytes) return AGG_ERR_INVALID_ARG;  // could never be admitted
  // staging with the smallest team it may get must fit the staging pool
  const uint32_t min_team = std::min<uint32_t>(8, (uint32_t)s->ki.blocks);
  if (plan_query(s, *q, min_team).stg_len > s->stage.bytes) return AGG_ERR_INVALID_ARG;
  {
    DeviceGuard g(s->device);
    const agg_status io = check_device_io(s->spec.ops, s->spec.value_type, q->d_keys, q->d_vals, q->n, &q->out, false);
    if (io != AGG_OK) return io;
  }
  const uint64_t t = s->next_ticket++;
  ServerQuery& sq = s->queries[t];
  sq.q = *q;
  sq.info.state = AGG_QUERY_QUEUED;
  sq.info.t_submit = s->now();
  s->waiting.push_back(t);
  s->submitted += 1;
  *ticket = t;
  return AGG_OK;
}

agg_status agg_server_progress(agg_server* s, uint32_t* completed) {
  if (!s) return AGG_ERR_INVALID_ARG;
  DeviceGuard g(s->device);
  uint32_t done = 0;
  for (size_t slot = 0; slot < s->slot_ticket.size(); ++slot) {
    if (s->slot_ticket[slot] < 0) continue;
    const cudaError_t e = cudaEventQuery(s->events[slot]);
    if (e == cudaErrorNotReady) continue;
    ServerQuery& sq = s->queries[(uint64_t)s->slot_ticket[slot]];
    sq.info.t_done = s->now();
    if (e != cudaSuccess) {
      cudaGetLastError();
      sq.info.state = AGG_QUERY_FAILED;
      sq.info.status = AGG_ERR_CUDA;
    } else {
      const unsigned long long bits = s->pinned[2 * slot];
      sq.info.status = status_from_bits(bits);
      sq.info.state = sq.info.status == AGG_OK ? AGG_QUERY_DONE : AGG_QUERY_FAILED;
      sq.info.n_groups = s->pinned[2 * slot + 1];
    }
    release_query(s, sq);
    s->slot_ticket[slot] = -1;
    s->running -= 1;
    s->completed += 1;
    ++done;
  }
  // Admission in arrival order.  A query needs a free slot, room in the pool
  // for its declared budget, room in the staging pool when it may spill, and
  // thread blocks: the teams of running queries never add up to more blocks
  // than the GPU holds at once, so that their cooperative grids never wait on
  // one another.  A query gets the blocks it wants, or fewer (at least
  // min(8, wanted)) when fewer are free.  Big queries (more than SMALL_TEAM
  // blocks wanted) share all but a reserve of the blocks and are admitted in
  // arrival order among themselves; a big query that must wait for blocks does
  // not hold back the small queries behind it.  A query that must wait for
  // memory holds back everything behind it, so that a large budget is never
  // starved.
  const uint32_t all = (uint32_t)s->ki.blocks;
  const uint32_t big_cap = s->slot_ticket.size() == 1 ? all : all - all / SMALL_RESERVE_DIV;
  bool big_blocked = false;
  for (auto it = s->waiting.begin(); it != s->waiting.end();) {
    int slot = -1;
    for (size_t i = 0; i < s->slot_ticket.size(); ++i)
      if (s->slot_ticket[i] < 0) {
        slot = (int)i;
        break;
      }
    if (slot < 0) break;
    const uint64_t t = *it;
    ServerQuery& sq = s->queries[t];
    // A query that fits its table at once runs on the in-budget kernels:
    // ordinary launches that wait on nothing and hold no team.
    const QueryPlan P0 = plan_query(s, sq.q, 0);
    const bool in_budget = P0.in_budget != 0 || P0.sort;
    const uint32_t want = in_budget ? 0u : team_wanted(sq.q.n, all, (uint32_t)s->slot_ticket.size());
    const bool big = want > SMALL_TEAM && s->slot_ticket.size() > 1;
    uint32_t avail = all - s->blocks_in_use;
    if (big) avail = std::min(avail, big_cap - std::min(big_cap, s->big_blocks_in_use));
    const uint32_t team = std::min(want, avail);
    if (!in_budget && ((big && big_blocked) || team < std::min(want, 8u))) {
      if (big) big_blocked = true;
      ++it;
      continue;
    }
    QueryPlan P = plan_query(s, sq.q, team);
    // a spilling query reserves one open staging chunk per block and partition:
    // a smaller team when that would not fit the staging pool at all
    for (uint32_t tm = team; P.stg_len > s->stage.bytes && tm > 8;) {
      tm /= 2;
      P = plan_query(s, sq.q, tm);
    }
    uint64_t off = 0, soff = 0;
    if (!pool_alloc(s->pool, P.L.total, &off)) break;
    if (!pool_alloc(s->stage, P.stg_len, &soff)) {
      pool_free(s->pool, off, P.L.total);
      break;
    }
    it = s->waiting.erase(it);
    sq.pool_off = off;
    sq.pool_len = P.L.total;
    sq.stg_off = soff;
    sq.stg_len = P.stg_len;
    sq.team = P.team;
    s->blocks_in_use += P.team;
    if (P.team > SMALL_TEAM) s->big_blocks_in_use += P.team;
    sq.slot = slot;
    const agg_status st = server_launch(s, sq, P, slot);
    sq.info.t_start = s->now();
    if (st != AGG_OK) {
      cudaGetLastError();
      // work queued before the failure may still use the ranges: let it drain
      cudaStreamSynchronize(s->streams[slot]);
      cudaGetLastError();
      release_query(s, sq);
      sq.info.state = AGG_QUERY_FAILED;
      sq.info.status = st;
      sq.info.t_done = s->now();
      s->completed += 1;
      continue;
    }
    sq.info.state = AGG_QUERY_RUNNING;
    s->slot_ticket[slot] = (int64_t)t;
    s->running += 1;
    s->max_conc = std::max<uint64_t>(s->max_conc, s->running);
  }
  if (completed) *completed = done;
  return AGG_OK;
}

agg_status agg_server_poll(agg_server* s, uint64_t ticket, agg_query_info* info) {
  if (!s || !info) return AGG_ERR_INVALID_ARG;
  auto it = s->queries.find(ticket);
  if (it == s->queries.end()) return AGG_ERR_INVALID_ARG;
  *info = it->second.info;
  return AGG_OK;
}

agg_status agg_server_get_stats(agg_server* s, agg_server_stats* st) {
  if (!s || !st) return AGG_ERR_INVALID_ARG;
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->running = s->running;
  st->queued = s->waiting.size();
  st->pool_bytes = s->pool.bytes;
  st->pool_in_use = s->pool.in_use;
  st->pool_peak = s->pool.peak;
  st->max_concurrent = s->max_conc;
  st->staging_bytes = s->stage.bytes;
  st->staging_in_use = s->stage.in_use;
  st->staging_peak = s->stage.peak;
  st->blocks = (uint64_t)s->ki.blocks;
  st->blocks_in_use = s->blocks_in_use;
  return AGG_OK;
}

agg_status agg_server_destroy(agg_server* s) {
  if (!s) return AGG_OK;
  DeviceGuard g(s->device);
  for (cudaStream_t st : s->streams)
    if (st) cudaStreamSynchronize(st);
  cudaGetLastError();
  for (cudaEvent_t e : s->events)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t st : s->streams)
    if (st) cudaStreamDestroy(st);
  if (s->mem) cudaFree(s->mem);
  if (s->pinned) cudaFreeHost(s->pinned);
  delete s;
  return AGG_OK;
}

}  // extern "C"
