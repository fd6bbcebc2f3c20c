// agg_run_noalloc: the in-budget hash group-by for callers that cannot allocate
// device memory.
//
// Some callers must not call cudaMalloc or cudaFree at all: code that runs
// inside a framework which owns every device allocation (a plug-in that is
// handed buffers and nothing else), code on a latency-critical path where an
// allocation (or the device-wide synchronisation a cudaFree implies) cannot be
// tolerated, and code that runs where no allocator is available.  They pass
// their input and output buffers; the working memory of the group-by (control
// block, tag bytes and table entries) lives in the file-scope array below,
// which every GPU that loads this library holds until the process exits.
//
// The array has room for AGG_NOALLOC_SLOTS table slots; inputs are limited to
// AGG_NOALLOC_MAX_ROWS rows, at most a quarter of the slots.  The group-by runs
// on the in-budget path: rows are split by hash into partitions that blocks
// aggregate in shared memory, and a key that does not fit there probes linearly
// across the table's active slots, so every distinct key finds a place whatever
// its hash (even for key sets built to collide) and nothing ever needs a
// staging area.  The partitions' scratch records use the top of the entries.
// All calls share the one array: calls whose work overlaps on the GPU race on
// it and must be ordered by the caller (one stream, or events).
#include <mutex>

#include "agg_internal.cuh"

namespace agg {
namespace {

constexpr uint32_t NA_SLOTS = AGG_NOALLOC_SLOTS;
constexpr uint64_t NA_CTRL = (sizeof(Ctrl) + 255) / 256 * 256;
constexpr uint64_t NA_TAGS = (NA_SLOTS + BUCKET + 255) / 256 * 256;
constexpr uint64_t NA_ENTRY = 64;  // the largest entry layout
constexpr uint64_t NA_BYTES = NA_CTRL + NA_TAGS + (uint64_t)(NA_SLOTS + 1) * NA_ENTRY;
static_assert(AGG_NOALLOC_MAX_ROWS * 4 <= AGG_NOALLOC_SLOTS, "rows must keep the table at most a quarter full");

// The scratch memory of agg_run_noalloc (control block, tags, entries).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct DeviceSetup {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  KernelInfo ki[3][2] = {};       // per entry layout and value type
};

constexpr int MAX_DEVICES = 64;
DeviceSetup g_setup[MAX_DEVICES];
std::mutex g_setup_mutex;

int entry_kind(uint32_t ops, int32_t vt) {
  if ((ops & (AGG_MIN | AGG_MAX)) == 0) return ENT32_CS;
  return vt == AGG_I32 ? ENT32_CSMM32 : ENT64;
}

// Once per device, with that device current: the device address of the scratch
// array (host code may not use the array's name as a device pointer) and the
// kernel's launch configuration.  Nothing is allocated.
agg_status setup_device(int dev, DeviceSetup** out) {
  if (dev < 0 || dev >= MAX_DEVICES) return AGG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& d = g_setup[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return AGG_ERR_CUDA;
    }
    d.base = static_cast<unsigned char*>(ptr);
    for (int ent = 0; ent < 3; ++ent)
      for (int vt = 0; vt < 2; ++vt) {
        if (ent == ENT32_CSMM32 && vt == AGG_I64) continue;
        if (hash_kernel_info(ent, vt, 2048, dev, &d.ki[ent][vt]) != cudaSuccess) {
          cudaGetLastError();
          return AGG_ERR_CUDA;
        }
      }
    d.ready = true;
  }
  *out = &d;
  return AGG_OK;
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace agg

using namespace agg;

extern "C" agg_status agg_run_noalloc(const agg_spec* spec, const int64_t* d_keys, const void* d_vals, uint64_t n,
                                      const agg_output* out, uint64_t* n_groups, void* stream) {
  if (!spec || !out || spec->ops == 0 || (spec->ops & ~15u) || spec->flags != 0 ||
      (spec->value_type != AGG_I32 && spec->value_type != AGG_I64) || spec->path != AGG_PATH_HASH)
    return AGG_ERR_INVALID_ARG;
  if (n > AGG_NOALLOC_MAX_ROWS) return AGG_ERR_INVALID_ARG;  // beyond the fixed scratch array
  const bool need_vals = (spec->ops & ~(uint32_t)AGG_COUNT) != 0;
  if (n > 0 && (!on_device(d_keys) || (need_vals && !on_device(d_vals)) || (d_vals && !on_device(d_vals))))
    return AGG_ERR_INVALID_ARG;
  if (!on_device(out->keys) || ((spec->ops & AGG_COUNT) && !on_device(out->count)) ||
      ((spec->ops & AGG_SUM) && !on_device(out->sum)) || ((spec->ops & AGG_MIN) && !on_device(out->min)) ||
      ((spec->ops & AGG_MAX) && !on_device(out->max)) || (out->d_n_groups && !on_device(out->d_n_groups)))
    return AGG_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_keys) & 7) ||
      (d_vals && (reinterpret_cast<uintptr_t>(d_vals) & (spec->value_type == AGG_I64 ? 7 : 3))))
    return AGG_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  DeviceSetup* d = nullptr;
  agg_status st = setup_device(dev, &d);
  if (st != AGG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ent = entry_kind(spec->ops, spec->value_type);
  // n <= AGG_NOALLOC_MAX_ROWS, a quarter of the slots: an in-budget path always
  // applies (the partitioned one, whose scratch sits at the top of the entries,
  // or for n = 0 the plain one, which then only publishes the empty result)
  const uint32_t es = entry_bytes(ent);
  PartPlan pp;
  const bool part = hash_part_plan(n, NA_SLOTS, es, 2048, &pp);
  const uint32_t s_act = part ? pp.s_ovf : hash_fast_slots(n, NA_SLOTS);
  if (s_act == 0) return AGG_ERR_INTERNAL;
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(d->base);
  uint32_t* tags = reinterpret_cast<uint32_t*>(d->base + NA_CTRL);
  uint8_t* ents = d->base + NA_CTRL + NA_TAGS;
  // The array keeps the previous call's contents: clear the control block and
  // the part of the table this call uses (its s_act slots, then the side slot
  // of the empty-marker key right after them).
  if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s) != cudaSuccess ||
      hash_init_table(ents, tags, s_act, ent, s) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  HashParams p{};
  p.keys = d_keys;
  p.vals = d_vals;
  p.n = n;
  p.has_vals = d_vals != nullptr;
  p.vec_ok = ((reinterpret_cast<uintptr_t>(d_keys) & 15) == 0) &&
             (!d_vals || (reinterpret_cast<uintptr_t>(d_vals) & (spec->value_type == AGG_I64 ? 15 : 7)) == 0);
  p.o_keys = out->keys;
  p.o_count = (spec->ops & AGG_COUNT) ? out->count : nullptr;
  p.o_sum = (spec->ops & AGG_SUM) ? out->sum : nullptr;
  p.o_min = (spec->ops & AGG_MIN) ? out->min : nullptr;
  p.o_max = (spec->ops & AGG_MAX) ? out->max : nullptr;
  p.o_cap = out->capacity;
  p.o_ngroups = out->d_n_groups;
  p.ctrl = ctrl;
  p.ent = ents;
  p.tags = tags;
  p.slots = s_act;  // the side slot follows the active slots
  p.seed = spec->seed;
  p.ops = spec->ops;
  p.fan_log2 = 4;
  p.lf = 0.5;
  p.s_act0 = s_act;
  p.ns = 2048;
  p.cache = 1;
  p.dedup = 0;
  p.timeout_ns = 4000000000ull;
  const size_t smem = d->ki[ent][spec->value_type].smem;
  if ((part ? hash_part_launch(ent, spec->value_type, p, pp, es, smem, s)
            : hash_fast_launch(ent, spec->value_type, p, s_act, smem, s)) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  // The run's status and group count, read in stream order on the caller's
  // stream (copies to pageable host memory return once they are complete).
  unsigned long long bits = 0, ng = 0;
  if (cudaMemcpyAsync(&bits, &ctrl->status_bits, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&ng, &ctrl->last_n_groups, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return AGG_ERR_CUDA;
  }
  if (n_groups) *n_groups = ng;
  if (bits & (1ull << (int)AGG_ERR_OUTPUT_CAPACITY)) return AGG_ERR_OUTPUT_CAPACITY;
  if (bits) return AGG_ERR_INTERNAL;
  return AGG_OK;
}
