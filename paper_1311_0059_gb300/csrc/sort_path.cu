// Sort path of the budgeted group-by (Section 4.1): radix sort + segmented reduction.
//
// The paper's Sort-based algorithm sorts memory-sized runs, merges them, and
// groups the merged stream with one running group.  Here the input is first
// split on the most significant bits of the (order-preserving) key into
// buckets that are stored in a staging area (outside the budget, like the
// paper's run files).  Consecutive buckets are gathered into rounds that fit
// the working-memory budget; each round is sorted on the full 64-bit key by an
// LSD radix sort with 8-bit digits, one "onesweep" pass per digit (Adinets and
// Merrill, 2022): each tile ranks its keys stably, publishes its digit counts,
// and obtains its global offsets by decoupled look-back over the preceding
// tiles.  Rounds are emitted in bucket order, so the output is in ascending
// signed key order.  The sorted round is then reduced segment by segment: a
// segment starts where the key changes, and each segment becomes one group
// record (COUNT, SUM, MIN, MAX).  A bucket too large for a round is split again
// on the next bits; a bucket holding a single key is reduced without sorting.
#include <algorithm>
#include <cstring>
#include <vector>

#include "sort_path.cuh"

namespace agg {
namespace {

constexpr int ST = 512;              // threads per block
constexpr int SIPT = 8;              // items per thread
constexpr int STILE = ST * SIPT;     // 4096 keys per tile
constexpr int SW = ST / 32;
constexpr int PASSES = 8;            // 8-bit digits over 64 bits
constexpr uint64_t MAX_ROUND = 8ull << 20;
constexpr unsigned FULLM = 0xFFFFFFFFu;
constexpr uint64_t SORT_TIMEOUT_NS = 4000000000ull;

constexpr uint64_t FLAG_AGG = 1, FLAG_INCL = 2;

__device__ __forceinline__ uint64_t ordkey(long long k) { return (uint64_t)k ^ 0x8000000000000000ull; }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t lanemask_lt_() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// status word of one (tile, digit): [epoch:32][flag:2][count:30]
__device__ __forceinline__ unsigned long long pack(uint32_t epoch, uint64_t flag, uint32_t count) {
  return ((unsigned long long)epoch << 32) | (flag << 30) | (unsigned long long)count;
}

__device__ __forceinline__ long long load_val(const void* v, int vt, uint64_t i) {
  return vt == AGG_I32 ? (long long)static_cast<const int*>(v)[i] : static_cast<const long long*>(v)[i];
}

// ---------------------------------------------------------------- MSD split

// Histogram of `nb` bits starting at `shift` over keys[0..n); also the key
// range (min, max of the order-preserving key) to detect single-key buckets.
__global__ void __launch_bounds__(ST) msd_hist_kernel(const long long* __restrict__ keys, uint64_t n, int shift,
                                                      uint32_t nbins, unsigned long long* __restrict__ hist,
                                                      unsigned long long* __restrict__ range) {
  __shared__ unsigned int h[256];
  for (uint32_t b = threadIdx.x; b < 256; b += ST) h[b] = 0;
  __syncthreads();
  uint64_t lo = ~0ull, hi = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)ST + threadIdx.x; i < n; i += (uint64_t)gridDim.x * ST) {
    const uint64_t u = ordkey(keys[i]);
    atomicAdd(&h[(u >> shift) & (nbins - 1)], 1u);
    lo = u < lo ? u : lo;
    hi = u > hi ? u : hi;
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < nbins; b += ST)
    if (h[b]) atomicAdd(hist + b, (unsigned long long)h[b]);
  for (int o = 16; o; o >>= 1) {
    const uint64_t l2 = __shfl_xor_sync(FULLM, lo, o), h2 = __shfl_xor_sync(FULLM, hi, o);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(range, (unsigned long long)lo);
    atomicMax(range + 1, (unsigned long long)hi);
  }
}

// Scatters (key, value) rows into their buckets; cursor[b] starts at the
// bucket's offset.  Order inside a bucket is not preserved (it is re-sorted).
__global__ void __launch_bounds__(ST) msd_scatter_kernel(const long long* __restrict__ keys, const void* __restrict__ vals,
                                                         int vt, uint64_t n, int shift, uint32_t nbins,
                                                         unsigned long long* __restrict__ cursor,
                                                         long long* __restrict__ okeys, long long* __restrict__ ovals) {
  __shared__ unsigned int cnt[256];
  __shared__ unsigned long long base[256];
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t ntiles = (n + STILE - 1) / STILE;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (uint32_t b = threadIdx.x; b < 256; b += ST) cnt[b] = 0;
    __syncthreads();
    long long k[SIPT], v[SIPT];
    uint32_t bin[SIPT], rk[SIPT];
    bool ok[SIPT];
#pragma unroll
    for (int i = 0; i < SIPT; ++i) {
      const uint64_t g = t * STILE + (uint64_t)i * ST + threadIdx.x;
      ok[i] = g < n;
      k[i] = ok[i] ? keys[g] : 0;
      v[i] = ok[i] ? (vals ? load_val(vals, vt, g) : 0) : 0;
      bin[i] = (uint32_t)(ordkey(k[i]) >> shift) & (nbins - 1);
      const uint32_t vm = __ballot_sync(FULLM, ok[i]);
      rk[i] = 0;
      if (ok[i]) {
        const uint32_t pm = __match_any_sync(vm, bin[i]);
        const int ldr = __ffs(pm) - 1;
        uint32_t b0 = 0;
        if ((int)lane == ldr) b0 = atomicAdd(&cnt[bin[i]], (uint32_t)__popc(pm));
        b0 = __shfl_sync(pm, b0, ldr);
        rk[i] = b0 + __popc(pm & lanemask_lt_());
      }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nbins; b += ST)
      base[b] = cnt[b] ? atomicAdd(cursor + b, (unsigned long long)cnt[b]) : 0ull;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SIPT; ++i) {
      if (!ok[i]) continue;
      const unsigned long long d = base[bin[i]] + rk[i];
      okeys[d] = k[i];
      ovals[d] = v[i];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- LSD onesweep

// All eight digit histograms of keys[0..m) in one pass.
__global__ void __launch_bounds__(ST) lsd_upsweep_kernel(const long long* __restrict__ keys, uint64_t m,
                                                         unsigned int* __restrict__ hist /*[8][256]*/) {
  __shared__ unsigned int h[PASSES * 256];
  for (uint32_t b = threadIdx.x; b < PASSES * 256; b += ST) h[b] = 0;
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)ST + threadIdx.x; i < m; i += (uint64_t)gridDim.x * ST) {
    const uint64_t u = ordkey(keys[i]);
#pragma unroll
    for (int p = 0; p < PASSES; ++p) atomicAdd(&h[p * 256 + ((u >> (8 * p)) & 255)], 1u);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < PASSES * 256; b += ST)
    if (h[b]) atomicAdd(hist + b, h[b]);
}

// Exclusive scan of each digit histogram (one block).
__global__ void lsd_scan_kernel(unsigned int* __restrict__ hist) {
  if (threadIdx.x < PASSES) {
    unsigned int acc = 0;
    unsigned int* h = hist + threadIdx.x * 256;
    for (int d = 0; d < 256; ++d) {
      const unsigned int c = h[d];
      h[d] = acc;
      acc += c;
    }
  }
}

struct OnesweepSmem {
  unsigned int whist[SW][256];
  long long keys[STILE];
  long long vals[STILE];
  unsigned int dstart[256];
  unsigned long long prefix[256];
  unsigned int tile;
};

// One LSD pass: stable ranking inside the tile, decoupled look-back over
// preceding tiles for the global offsets, scatter through shared memory so
// that runs of equal digits are written contiguously.
__global__ void __launch_bounds__(ST) onesweep_kernel(const long long* __restrict__ ik, const void* __restrict__ iv,
                                                      int ivt, long long* __restrict__ ok, long long* __restrict__ ov,
                                                      uint64_t m, int pass, const unsigned int* __restrict__ gbase,
                                                      unsigned long long* __restrict__ status,
                                                      unsigned int* __restrict__ tile_ctr, uint32_t epoch,
                                                      unsigned long long* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char sraw[];
  OnesweepSmem& S = *reinterpret_cast<OnesweepSmem*>(sraw);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int shift = 8 * pass;
  if (threadIdx.x == 0) S.tile = atomicAdd(tile_ctr, 1u);
  for (uint32_t i = threadIdx.x; i < SW * 256; i += ST) (&S.whist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t tile = S.tile;
  const uint64_t t0 = (uint64_t)tile * STILE;
  const uint32_t tcount = (uint32_t)((m - t0) < (uint64_t)STILE ? (m - t0) : (uint64_t)STILE);

  long long k[SIPT], v[SIPT];
  uint32_t dg[SIPT], rk[SIPT];
  bool okk[SIPT];
  // warp w owns the contiguous range [w*32*SIPT, (w+1)*32*SIPT) of the tile
#pragma unroll
  for (int i = 0; i < SIPT; ++i) {
    const uint32_t li = warp * 32 * SIPT + i * 32 + lane;
    okk[i] = li < tcount;
    const uint64_t g = t0 + li;
    k[i] = okk[i] ? ik[g] : 0;
    v[i] = okk[i] ? (iv ? load_val(iv, ivt, g) : 0) : 0;
    dg[i] = (uint32_t)(ordkey(k[i]) >> shift) & 255u;
  }
#pragma unroll
  for (int i = 0; i < SIPT; ++i) {
    const uint32_t vm = __ballot_sync(FULLM, okk[i]);
    uint32_t peers = 0;
    if (okk[i]) peers = __match_any_sync(vm, dg[i]);
    rk[i] = okk[i] ? S.whist[warp][dg[i]] + __popc(peers & lanemask_lt_()) : 0;
    __syncwarp();
    if (okk[i] && (int)lane == __ffs(peers) - 1) S.whist[warp][dg[i]] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, tile count, publish, look back
  unsigned int cnt = 0;
  if (threadIdx.x < 256) {
    const uint32_t d = threadIdx.x;
    for (int w = 0; w < SW; ++w) {
      const unsigned int c = S.whist[w][d];
      S.whist[w][d] = cnt;
      cnt += c;
    }
    unsigned long long* my = status + (uint64_t)tile * 256 + d;
    if (tile == 0) {
      st_release_u64(my, pack(epoch, FLAG_INCL, cnt));
      S.prefix[d] = gbase[d];
    } else {
      st_release_u64(my, pack(epoch, FLAG_AGG, cnt));
      unsigned long long excl = 0;
      int64_t t = (int64_t)tile - 1;
      const uint64_t ts = globaltimer_ns();
      while (t >= 0) {
        const unsigned long long s = ld_acquire_u64(status + (uint64_t)t * 256 + d);
        const uint32_t ep = (uint32_t)(s >> 32);
        const uint64_t fl = (s >> 30) & 3;
        if (ep != epoch || fl == 0) {
          __nanosleep(32);
          if (globaltimer_ns() - ts > SORT_TIMEOUT_NS) {
            atomicOr(err, 1ull << (int)AGG_ERR_TIMEOUT);
            break;
          }
          continue;
        }
        excl += s & 0x3FFFFFFFull;
        if (fl == FLAG_INCL) break;
        --t;
      }
      st_release_u64(my, pack(epoch, FLAG_INCL, (uint32_t)(excl + cnt)));
      S.prefix[d] = gbase[d] + excl;
    }
  }
  // digit starts inside the tile (exclusive scan of the 256 tile counts)
  __shared__ unsigned int wsum[8];
  if (threadIdx.x < 256) {
    unsigned int inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(FULLM, inc, o);
      if ((int)lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    S.dstart[threadIdx.x] = inc - cnt;
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    unsigned int add = 0;
    for (uint32_t w = 0; w < warp; ++w) add += wsum[w];
    S.dstart[threadIdx.x] += add;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SIPT; ++i) {
    if (!okk[i]) continue;
    const uint32_t pos = S.dstart[dg[i]] + S.whist[warp][dg[i]] + rk[i];
    S.keys[pos] = k[i];
    S.vals[pos] = v[i];
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < tcount; j += ST) {
    const long long kk = S.keys[j];
    const uint32_t d = (uint32_t)(ordkey(kk) >> shift) & 255u;
    const unsigned long long dst = S.prefix[d] + (j - S.dstart[d]);
    ok[dst] = kk;
    ov[dst] = S.vals[j];
  }
}

// ---------------------------------------------------------------- segmented reduction

// Heads (positions where the key changes) per tile of STILE records.
__global__ void __launch_bounds__(ST) seg_heads_kernel(const long long* __restrict__ keys, uint64_t m,
                                                       unsigned int* __restrict__ heads) {
  const uint64_t t = blockIdx.x;
  const uint64_t t0 = t * STILE;
  unsigned int c = 0;
  for (uint32_t j = threadIdx.x; j < STILE; j += ST) {
    const uint64_t g = t0 + j;
    if (g < m && (g == 0 || keys[g] != keys[g - 1])) ++c;
  }
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(FULLM, c, o);
  __shared__ unsigned int ws[SW];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int s = 0;
    for (int w = 0; w < SW; ++w) s += ws[w];
    heads[t] = s;
  }
}

// Exclusive scan of head counts (one block), offset by the running group
// count; the running count then advances by this round's groups.
__global__ void seg_scan_kernel(const unsigned int* __restrict__ heads, uint32_t ntiles,
                                unsigned long long* __restrict__ tile_out, unsigned long long* __restrict__ run_base) {
  __shared__ unsigned long long part[1024];
  const uint32_t per = (ntiles + blockDim.x - 1) / blockDim.x;
  const uint32_t b = threadIdx.x * per;
  unsigned long long s = 0;
  for (uint32_t i = 0; i < per && b + i < ntiles; ++i) s += heads[b + i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long acc = *run_base;
    for (uint32_t i = 0; i < blockDim.x; ++i) {
      const unsigned long long c = part[i];
      part[i] = acc;
      acc += c;
    }
    *run_base = acc;
  }
  __syncthreads();
  unsigned long long acc = part[threadIdx.x];
  for (uint32_t i = 0; i < per && b + i < ntiles; ++i) {
    tile_out[b + i] = acc;
    acc += heads[b + i];
  }
}

struct SegOut {
  long long* keys;
  unsigned long long* count;
  long long* sum;
  long long* mn;
  long long* mx;
  uint64_t cap;
};

__device__ __forceinline__ void seg_write(const SegOut& o, uint64_t idx, long long key, unsigned long long c,
                                          unsigned long long s, long long mn, long long mx,
                                          unsigned long long* err) {
  if (idx >= o.cap) {
    atomicOr(err, 1ull << (int)AGG_ERR_OUTPUT_CAPACITY);
    return;
  }
  o.keys[idx] = key;
  if (o.count) o.count[idx] = c;
  if (o.sum) o.sum[idx] = (long long)s;
  if (o.mn) o.mn[idx] = mn;
  if (o.mx) o.mx[idx] = mx;
}

// Each head reduces its segment up to the tile end; the piece of a segment
// that continues from an earlier tile is left as this tile's carry.
__global__ void __launch_bounds__(ST) seg_reduce_kernel(const long long* __restrict__ keys,
                                                        const long long* __restrict__ vals, uint64_t m,
                                                        const unsigned long long* __restrict__ tile_out, SegOut o,
                                                        unsigned long long* __restrict__ carry /*[tiles][4]*/,
                                                        unsigned int* __restrict__ carry_ok,
                                                        unsigned long long* __restrict__ err) {
  const uint64_t t = blockIdx.x;
  const uint64_t t0 = t * STILE;
  const uint64_t tend = (t0 + STILE < m) ? t0 + STILE : m;
  // thread owns SIPT consecutive positions
  const uint64_t p0 = t0 + (uint64_t)threadIdx.x * SIPT;
  bool head[SIPT];
  unsigned int c = 0;
#pragma unroll
  for (int i = 0; i < SIPT; ++i) {
    const uint64_t g = p0 + i;
    head[i] = g < tend && (g == 0 || keys[g] != keys[g - 1]);
    c += head[i];
  }
  // block exclusive scan of head counts in position order
  __shared__ unsigned int ws[SW];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int inc = c;
  for (int o2 = 1; o2 < 32; o2 <<= 1) {
    const unsigned int y = __shfl_up_sync(FULLM, inc, o2);
    if ((int)lane >= o2) inc += y;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  unsigned int before = inc - c;
  for (uint32_t w = 0; w < warp; ++w) before += ws[w];
  uint64_t idx = tile_out[t] + before;
#pragma unroll 1
  for (int i = 0; i < SIPT; ++i) {
    if (!head[i]) continue;
    const uint64_t g = p0 + i;
    const long long key = keys[g];
    unsigned long long cn = 0, sm = 0;
    long long mn = INT64_MAX, mx = INT64_MIN;
    for (uint64_t j = g; j < tend && keys[j] == key; ++j) {
      const long long val = vals[j];
      ++cn;
      sm += (unsigned long long)val;
      mn = val < mn ? val : mn;
      mx = val > mx ? val : mx;
    }
    seg_write(o, idx, key, cn, sm, mn, mx, err);
    ++idx;
  }
  if (threadIdx.x == 0) {
    const bool cont = t0 > 0 && t0 < m && keys[t0] == keys[t0 - 1];
    carry_ok[t] = cont;
    if (cont) {
      const long long key = keys[t0];
      unsigned long long cn = 0, sm = 0;
      long long mn = INT64_MAX, mx = INT64_MIN;
      for (uint64_t j = t0; j < tend && keys[j] == key; ++j) {
        const long long val = vals[j];
        ++cn;
        sm += (unsigned long long)val;
        mn = val < mn ? val : mn;
        mx = val > mx ? val : mx;
      }
      carry[t * 4 + 0] = cn;
      carry[t * 4 + 1] = sm;
      carry[t * 4 + 2] = (unsigned long long)mn;
      carry[t * 4 + 3] = (unsigned long long)mx;
    }
  }
}

// Folds each tile's carry into the group that started before the tile.
__global__ void seg_fix_kernel(const unsigned long long* __restrict__ carry, const unsigned int* __restrict__ carry_ok,
                               const unsigned long long* __restrict__ tile_out, uint32_t ntiles, SegOut o) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles || !carry_ok[t]) return;
  const uint64_t idx = tile_out[t] - 1;
  if (idx >= o.cap) return;
  if (o.count) atomicAdd(o.count + idx, carry[t * 4 + 0]);
  if (o.sum) atomicAdd(reinterpret_cast<unsigned long long*>(o.sum) + idx, carry[t * 4 + 1]);
  if (o.mn) atomicMin(o.mn + idx, (long long)carry[t * 4 + 2]);
  if (o.mx) atomicMax(o.mx + idx, (long long)carry[t * 4 + 3]);
}

__global__ void sort_finish_kernel(const unsigned long long* __restrict__ run_base, uint64_t* o_ngroups, Ctrl* ctrl,
                                   uint64_t n, const unsigned long long* __restrict__ err) {
  const unsigned long long ng = *run_base;
  if (o_ngroups) *o_ngroups = ng;
  ctrl->last_n_rows = n;
  ctrl->last_n_groups = ng;
  ctrl->last_levels = 1;
  atomicOr(&ctrl->status_bits, *err);
}

// Reduction of a segment whose keys are all equal (no sort needed).
__global__ void __launch_bounds__(ST) single_key_kernel(const void* __restrict__ vals, int vt, uint64_t n,
                                                        unsigned long long* __restrict__ acc /*[4]*/) {
  unsigned long long c = 0, sm = 0;
  long long mn = INT64_MAX, mx = INT64_MIN;
  for (uint64_t i = blockIdx.x * (uint64_t)ST + threadIdx.x; i < n; i += (uint64_t)gridDim.x * ST) {
    const long long v = vals ? load_val(vals, vt, i) : 0;
    ++c;
    sm += (unsigned long long)v;
    mn = v < mn ? v : mn;
    mx = v > mx ? v : mx;
  }
  for (int o = 16; o; o >>= 1) {
    c += __shfl_xor_sync(FULLM, c, o);
    sm += __shfl_xor_sync(FULLM, sm, o);
    const long long a = __shfl_xor_sync(FULLM, mn, o), b = __shfl_xor_sync(FULLM, mx, o);
    mn = a < mn ? a : mn;
    mx = b > mx ? b : mx;
  }
  if ((threadIdx.x & 31) == 0 && c) {
    atomicAdd(acc + 0, c);
    atomicAdd(acc + 1, sm);
    atomicMin(reinterpret_cast<long long*>(acc + 2), mn);
    atomicMax(reinterpret_cast<long long*>(acc + 3), mx);
  }
}

__global__ void single_key_write_kernel(const long long* __restrict__ keys, const unsigned long long* __restrict__ acc,
                                        unsigned long long* __restrict__ run_base, SegOut o,
                                        unsigned long long* __restrict__ err) {
  const unsigned long long idx = *run_base;
  seg_write(o, idx, keys[0], acc[0], acc[1], (long long)acc[2], (long long)acc[3], err);
  *run_base = idx + 1;
}

// ---------------------------------------------------------------- host driver

struct Work {
  long long* ak;
  long long* av;
  long long* bk;
  long long* bv;
  unsigned long long* status;  // [max_tiles][256]
  unsigned int* hist;          // [8][256]
  unsigned int* tile_ctr;      // [8]
  unsigned long long* run_base;
  unsigned long long* err;
  unsigned long long* msd_hist;  // [256]
  unsigned long long* range;     // [2]
  unsigned long long* cursor;    // [256]
  unsigned int* heads;           // [max_tiles]
  unsigned long long* tile_out;  // [max_tiles]
  unsigned long long* carry;     // [max_tiles][4]
  unsigned int* carry_ok;        // [max_tiles]
};

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

uint64_t work_bytes_for(uint64_t rows) {
  const uint64_t tiles = (rows + STILE - 1) / STILE + 1;
  uint64_t b = 0;
  b += 4 * align256(rows * 8);                // two double buffers of keys and values
  b += align256(tiles * 256 * 8);             // look-back status
  b += align256(PASSES * 256 * 4) + align256(PASSES * 4) + 3 * 256;
  b += align256(256 * 8) + align256(16) + align256(256 * 8);
  b += align256(tiles * 4) + align256(tiles * 8) + align256(tiles * 32) + align256(tiles * 4);
  return b + 4096;
}

Work carve(void* base, uint64_t rows) {
  const uint64_t tiles = (rows + STILE - 1) / STILE + 1;
  uint8_t* p = static_cast<uint8_t*>(base);
  auto take = [&](uint64_t bytes) {
    uint8_t* r = p;
    p += align256(bytes);
    return r;
  };
  Work w;
  w.ak = reinterpret_cast<long long*>(take(rows * 8));
  w.av = reinterpret_cast<long long*>(take(rows * 8));
  w.bk = reinterpret_cast<long long*>(take(rows * 8));
  w.bv = reinterpret_cast<long long*>(take(rows * 8));
  w.status = reinterpret_cast<unsigned long long*>(take(tiles * 256 * 8));
  w.hist = reinterpret_cast<unsigned int*>(take(PASSES * 256 * 4));
  w.tile_ctr = reinterpret_cast<unsigned int*>(take(PASSES * 4));
  w.run_base = reinterpret_cast<unsigned long long*>(take(256));
  w.err = reinterpret_cast<unsigned long long*>(take(256));
  w.msd_hist = reinterpret_cast<unsigned long long*>(take(256 * 8));
  w.range = reinterpret_cast<unsigned long long*>(take(256));
  w.cursor = reinterpret_cast<unsigned long long*>(take(256 * 8));
  w.heads = reinterpret_cast<unsigned int*>(take(tiles * 4));
  w.tile_out = reinterpret_cast<unsigned long long*>(take(tiles * 8));
  w.carry = reinterpret_cast<unsigned long long*>(take(tiles * 32));
  w.carry_ok = reinterpret_cast<unsigned int*>(take(tiles * 4));
  return w;
}

struct Driver {
  SortState& s;
  Work w;
  SegOut o;
  cudaStream_t st;
  int sms;
  uint64_t round_rows;
  bool failed = false;

  bool ok(cudaError_t e) {
    if (e != cudaSuccess) {
      cudaGetLastError();
      failed = true;
    }
    return !failed;
  }
  unsigned grid_for(uint64_t n, unsigned per_sm) {
    uint64_t b = (n + ST - 1) / ST;
    const uint64_t cap = (uint64_t)sms * per_sm;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
  }

  // Reduces records [0, m) of (keys, vals), already sorted (or single-key).
  void reduce(const long long* keys, const long long* vals, uint64_t m) {
    const uint32_t tiles = (uint32_t)((m + STILE - 1) / STILE);
    seg_heads_kernel<<<tiles, ST, 0, st>>>(keys, m, w.heads);
    seg_scan_kernel<<<1, 1024, 0, st>>>(w.heads, tiles, w.tile_out, w.run_base);
    seg_reduce_kernel<<<tiles, ST, 0, st>>>(keys, vals, m, w.tile_out, o, w.carry, w.carry_ok, w.err);
    seg_fix_kernel<<<(tiles + 255) / 256, 256, 0, st>>>(w.carry, w.carry_ok, w.tile_out, tiles, o);
    s.launches += 4;
    ok(cudaGetLastError());
  }

  // Sorts records [0, m) (m <= round_rows) on the full key into buffer A or B
  // and reduces them.  Source values may be int32 (the caller's input).
  void sort_round(const long long* keys, const void* vals, int vt, uint64_t m) {
    if (m == 0) return;
    ok(cudaMemsetAsync(w.hist, 0, PASSES * 256 * 4, st));
    ok(cudaMemsetAsync(w.tile_ctr, 0, PASSES * 4, st));
    lsd_upsweep_kernel<<<grid_for(m, 2), ST, 0, st>>>(keys, m, w.hist);
    lsd_scan_kernel<<<1, 32, 0, st>>>(w.hist);
    s.launches += 2;
    const long long* ik = keys;
    const void* iv = vals;
    int ivt = vt;
    const uint32_t tiles = (uint32_t)((m + STILE - 1) / STILE);
    for (int p = 0; p < PASSES; ++p) {
      long long* okey = (p & 1) ? w.bk : w.ak;
      long long* oval = (p & 1) ? w.bv : w.av;
      const uint32_t epoch = ++s.epoch;
      onesweep_kernel<<<tiles, ST, sizeof(OnesweepSmem), st>>>(ik, iv, ivt, okey, oval, m, p, w.hist + p * 256,
                                                               w.status, w.tile_ctr + p, epoch, w.err);
      s.launches += 1;
      ik = okey;
      iv = oval;
      ivt = AGG_I64;
    }
    ok(cudaGetLastError());
    s.last_passes += PASSES;
    s.last_rounds += 1;
    reduce(ik, static_cast<const long long*>(iv), m);
  }

  // Splits [0, n) on `nb` bits below `fixed` key bits and processes the
  // buckets in key order.  `depth` > 0 allocates its own staging.
  void split(const long long* keys, const void* vals, int vt, uint64_t n, int fixed, int depth) {
    if (failed || n == 0) return;
    // single-key segment: reduce as is
    ok(cudaMemsetAsync(w.msd_hist, 0, 256 * 8, st));
    unsigned long long rinit[2] = {~0ull, 0ull};
    ok(cudaMemcpyAsync(w.range, rinit, 16, cudaMemcpyHostToDevice, st));
    int nb = 1;
    while (nb < 8 && ((n >> nb) > round_rows / 2)) ++nb;
    if (nb > 64 - fixed) nb = 64 - fixed;
    const int shift = 64 - fixed - nb;
    msd_hist_kernel<<<grid_for(n, 4), ST, 0, st>>>(keys, n, shift, 1u << nb, w.msd_hist, w.range);
    s.launches += 1;
    std::vector<unsigned long long> h(256), rg(2);
    if (!ok(cudaMemcpyAsync(h.data(), w.msd_hist, 256 * 8, cudaMemcpyDeviceToHost, st))) return;
    if (!ok(cudaMemcpyAsync(rg.data(), w.range, 16, cudaMemcpyDeviceToHost, st))) return;
    if (!ok(cudaStreamSynchronize(st))) return;
    if (rg[0] == rg[1]) {  // one distinct key: reduce without sorting
      ok(cudaMemsetAsync(w.carry, 0, 32, st));
      const unsigned long long init[4] = {0ull, 0ull, (unsigned long long)INT64_MAX, (unsigned long long)INT64_MIN};
      ok(cudaMemcpyAsync(w.carry, init, 32, cudaMemcpyHostToDevice, st));
      single_key_kernel<<<grid_for(n, 4), ST, 0, st>>>(vals, vt, n, w.carry);
      single_key_write_kernel<<<1, 1, 0, st>>>(keys, w.carry, w.run_base, o, w.err);
      s.launches += 2;
      ok(cudaGetLastError());
      s.last_buckets += 1;
      return;
    }
    const uint32_t nbins = 1u << nb;
    std::vector<unsigned long long> off(nbins + 1, 0);
    for (uint32_t b = 0; b < nbins; ++b) off[b + 1] = off[b] + h[b];
    void* mem = nullptr;
    long long* sk;
    long long* sv;
    if (depth == 0) {
      sk = static_cast<long long*>(s.mem);
      sv = sk + s.reserved_rows;
    } else {
      if (!ok(cudaMallocAsync(&mem, n * 16, st))) return;
      sk = static_cast<long long*>(mem);
      sv = sk + n;
    }
    ok(cudaMemcpyAsync(w.cursor, off.data(), nbins * 8, cudaMemcpyHostToDevice, st));
    msd_scatter_kernel<<<grid_for(n, 2), ST, 0, st>>>(keys, vals, vt, n, shift, nbins, w.cursor, sk, sv);
    s.launches += 1;
    ok(cudaGetLastError());
    s.last_levels = std::max<uint64_t>(s.last_levels, (uint64_t)depth + 1);
    // rounds: consecutive buckets while they fit
    uint32_t b = 0;
    while (b < nbins && !failed) {
      if (h[b] == 0) {
        ++b;
        continue;
      }
      if (h[b] > round_rows) {
        split(sk + off[b], sv + off[b], AGG_I64, h[b], fixed + nb, depth + 1);
        ++b;
        continue;
      }
      uint32_t e = b;
      uint64_t tot = 0;
      while (e < nbins && h[e] <= round_rows && tot + h[e] <= round_rows) {
        tot += h[e];
        ++e;
      }
      s.last_buckets += (e - b);
      sort_round(sk + off[b], sv + off[b], AGG_I64, tot);
      b = e;
    }
    if (mem) cudaFreeAsync(mem, st);
  }

};

uint64_t rows_fitting(uint64_t avail) {
  uint64_t lo = 0, hi = MAX_ROUND;
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) / 2;
    if (work_bytes_for(mid) <= avail) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

uint64_t round_rows_for(size_t budget) {
  // largest round whose working memory fits the budget (minus the control block)
  const uint64_t avail = budget > 65536 ? budget - 65536 : 0;
  uint64_t lo = 0, hi = MAX_ROUND;
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) / 2;
    if (work_bytes_for(mid) <= avail) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

}  // namespace

uint64_t sort_rows_for(uint64_t work_bytes) { return rows_fitting(work_bytes); }

void sort_attach(SortState& s, void* work, uint64_t work_bytes) {
  s.work = work;
  s.work_bytes = work_bytes;
  s.round_rows = rows_fitting(work_bytes);
  s.external = true;
  cudaFuncSetAttribute(reinterpret_cast<const void*>(&onesweep_kernel), cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(OnesweepSmem));
}

agg_status sort_reserve(SortState& s, uint64_t rows, size_t budget, const agg_spec&) {
  // `budget` here is what remains of the handle's budget after its control block
  if (s.external && s.round_rows < STILE) return AGG_ERR_BUDGET_TOO_SMALL;
  if (!s.work) {
    const uint64_t rr = round_rows_for(budget);
    if (rr < STILE) return AGG_ERR_BUDGET_TOO_SMALL;
    const uint64_t wb = work_bytes_for(rr);
    if (cudaMalloc(&s.work, wb) != cudaSuccess) {
      cudaGetLastError();
      s.work = nullptr;
      return AGG_ERR_OOM;
    }
    if (cudaMemset(s.work, 0, wb) != cudaSuccess) {
      cudaGetLastError();
      return AGG_ERR_CUDA;
    }
    s.work_bytes = wb;
    s.round_rows = rr;
    cudaFuncSetAttribute(reinterpret_cast<const void*>(&onesweep_kernel), cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(OnesweepSmem));
  }
  if (rows > s.round_rows && rows > s.reserved_rows) {
    if (s.mem) cudaFree(s.mem);
    s.mem = nullptr;
    s.mem_bytes = 0;
    s.reserved_rows = 0;
    if (cudaMalloc(&s.mem, rows * 16) != cudaSuccess) {
      cudaGetLastError();
      s.mem = nullptr;
      return AGG_ERR_OOM;
    }
    s.mem_bytes = rows * 16;
    s.reserved_rows = rows;
  }
  return AGG_OK;
}

agg_status sort_run(SortState& s, size_t budget, const agg_spec& spec, Ctrl* ctrl, const int64_t* d_keys,
                    const void* d_vals, uint64_t n, const agg_output* out, cudaStream_t stream) {
  agg_status st = sort_reserve(s, n, budget, spec);
  if (st != AGG_OK) return st;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  Driver d{s, carve(s.work, s.round_rows), {}, stream, sms, s.round_rows};
  d.o.keys = reinterpret_cast<long long*>(out->keys);
  d.o.count = (spec.ops & AGG_COUNT) ? reinterpret_cast<unsigned long long*>(out->count) : nullptr;
  d.o.sum = (spec.ops & AGG_SUM) ? reinterpret_cast<long long*>(out->sum) : nullptr;
  d.o.mn = (spec.ops & AGG_MIN) ? reinterpret_cast<long long*>(out->min) : nullptr;
  d.o.mx = (spec.ops & AGG_MAX) ? reinterpret_cast<long long*>(out->max) : nullptr;
  d.o.cap = out->capacity;
  s.last_buckets = s.last_passes = s.last_rounds = s.last_levels = 0;
  d.ok(cudaMemsetAsync(d.w.run_base, 0, 8, stream));
  d.ok(cudaMemsetAsync(d.w.err, 0, 8, stream));
  if (s.external)  // memory another path used: no stale look-back word may match an epoch
    d.ok(cudaMemsetAsync(d.w.status, 0, ((s.round_rows + STILE - 1) / STILE + 1) * 256 * 8, stream));
  const long long* keys = reinterpret_cast<const long long*>(d_keys);
  if (n > 0) {
    if (n <= s.round_rows) {
      s.last_buckets = 1;
      d.sort_round(keys, d_vals, spec.value_type, n);
    } else {
      d.split(keys, d_vals, spec.value_type, n, 0, 0);
    }
  }
  sort_finish_kernel<<<1, 1, 0, stream>>>(d.w.run_base, out->d_n_groups, ctrl, n, d.w.err);
  s.launches += 1;
  d.ok(cudaGetLastError());
  return d.failed ? AGG_ERR_CUDA : AGG_OK;
}

void sort_free(SortState& s) {
  if (s.mem) cudaFree(s.mem);
  if (s.work && !s.external) cudaFree(s.work);
  const uint64_t l = s.launches, e = s.epoch;
  s = SortState{};
  s.launches = l;
  s.epoch = e;
}

uint64_t sort_staging_bytes(const SortState& s) { return s.mem_bytes; }

void sort_fill_stats(const SortState& s, agg_stats* st) {
  st->levels = s.last_levels ? s.last_levels : 1;
  st->rounds = s.last_rounds;
  st->table_bytes = s.work_bytes;
  st->fan_out = s.last_buckets;
}

}  // namespace agg
