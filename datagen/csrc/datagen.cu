// Device implementation of the seeded synthetic-input generator.
//
// Produces exactly the bytes of the numpy definitions in datagen/__init__.py:
// SplitMix64 streams (Steele, Lea and Flood, OOPSLA 2014), a bijective
// rank -> key map, multiply-high uniform ranks, Zipf ranks by searching a
// host-built float64 CDF table, and the two value distributions.  It holds
// none of the group-by arithmetic.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;
constexpr uint64_t M1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t M2 = 0x94D049BB133111EBull;

__host__ __device__ inline uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * M1;
  z = (z ^ (z >> 27)) * M2;
  return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t stream_base(uint64_t seed, uint64_t sid) {
  return mix(seed ^ ((sid + 1) * GAMMA));
}

// floor(u * d / 2^64) for d < 2^32, by 32-bit halves (matches the numpy form).
__device__ inline uint64_t mulhi_u32(uint64_t u, uint64_t d) {
  uint64_t hi = (u >> 32) * d;
  uint64_t lo = ((u & 0xFFFFFFFFull) * d) >> 32;
  return (hi + lo) >> 32;
}

__global__ void gen_rows_kernel(uint64_t seed, uint64_t domain, int dist, const double* __restrict__ cdf,
                                int vtype, uint64_t start, uint64_t count, int64_t* __restrict__ keys,
                                void* __restrict__ vals) {
  const uint64_t kb = stream_base(seed, 0);
  const uint64_t vb = stream_base(seed, 1);
  const uint64_t salt = mix(stream_base(seed, 2) + GAMMA);
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < count;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = start + j;
    const uint64_t u = mix(kb + (i + 1) * GAMMA);
    uint64_t rank;
    if (dist == 0) {
      rank = mulhi_u32(u, domain);
    } else {
      const double t = (double)(u >> 11) * 0x1p-53;
      uint64_t lo = 0, hi = domain - 1;  // cdf[domain-1] == 2.0 > t
      while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (cdf[mid] > t) hi = mid; else lo = mid + 1;
      }
      rank = lo;
    }
    if (keys) keys[j] = (int64_t)mix(rank ^ salt);
    if (vals) {
      const uint64_t w = mix(vb + (i + 1) * GAMMA);
      if (vtype == 0) static_cast<int32_t*>(vals)[j] = (int32_t)mulhi_u32(w, 1000);
      else static_cast<int64_t*>(vals)[j] = (int64_t)(w >> 44);
    }
  }
}

}  // namespace

extern "C" int datagen_rows(uint64_t seed, uint64_t domain, int dist, const void* cdf, int vtype, uint64_t start,
                            uint64_t count, void* keys, void* vals, void* stream) {
  if (count == 0) return 0;
  if (domain == 0 || domain >= (1ull << 32)) return (int)cudaErrorInvalidValue;
  if (dist == 1 && cdf == nullptr) return (int)cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t blocks = (count + 255) / 256;
  uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * 16;
  if (blocks > cap) blocks = cap;
  gen_rows_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
      seed, domain, dist, static_cast<const double*>(cdf), vtype, start, count, static_cast<int64_t*>(keys), vals);
  return (int)cudaGetLastError();
}
