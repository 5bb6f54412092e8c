// Device helpers shared by the two Delta-stepping engines (og_kernels.cu, og_async.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "og_internal.cuh"

namespace og {

#define FULL 0xffffffffu

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// A* heuristic floor(100 * Euclidean distance to the target).  Integral coordinates:
// exact integer square root of 10000 * (dx^2 + dy^2) (double estimate, then corrected
// so that s^2 <= N < (s+1)^2).  Otherwise a double evaluation minus one unit, which stays
// below the exact value.
__device__ __forceinline__ uint32_t heuristic(const float2* xy, uint32_t integral, uint32_t v,
                                              float tx, float ty) {
  const float2 p = __ldg(xy + v);
  if (integral) {
    const long long dx = (long long)p.x - (long long)tx;
    const long long dy = (long long)p.y - (long long)ty;
    const unsigned long long N = 10000ull * (unsigned long long)(dx * dx + dy * dy);
    unsigned long long s = (unsigned long long)sqrt((double)N);
    while (s * s > N) --s;
    while ((s + 1) * (s + 1) <= N) ++s;
    return s >= kSat ? kSat - 1 : (uint32_t)s;
  }
  const double dx = (double)p.x - (double)tx, dy = (double)p.y - (double)ty;
  const double d = floor(100.0 * sqrt(dx * dx + dy * dy)) - 1.0;
  if (!(d > 0.0)) return 0u;
  return d >= 4.0e9 ? 4000000000u : (uint32_t)d;
}

constexpr int kEllWidth = 8;  // edges per ELL row (64 bytes)

// Brings a vertex's adjacency into L2 ahead of its expansion.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_row(const uint4* ell, const uint32_t* off, uint32_t v) {
  if (ell) {
    const uint4* r = ell + (size_t)v * 4;
    prefetch_l2(r);
    prefetch_l2(r + 2);
  } else {
    prefetch_l2(off + v);
  }
}

// Loads one ELL row: up to 8 {neighbor, weight} pairs in four 16-byte loads.
__device__ __forceinline__ void load_row(const uint4* ell, uint32_t v, uint2 (&ew)[kEllWidth]) {
  const uint4* r = ell + (size_t)v * 4;
  const uint4 a = __ldg(r), b = __ldg(r + 1), c = __ldg(r + 2), d = __ldg(r + 3);
  ew[0] = make_uint2(a.x, a.y); ew[1] = make_uint2(a.z, a.w);
  ew[2] = make_uint2(b.x, b.y); ew[3] = make_uint2(b.z, b.w);
  ew[4] = make_uint2(c.x, c.y); ew[5] = make_uint2(c.z, c.w);
  ew[6] = make_uint2(d.x, d.y); ew[7] = make_uint2(d.z, d.w);
}

// Cached read of a distance for the pre-check: a stale copy can only be larger than the
// current value, so "new >= cached" proves the relaxation cannot improve.
__device__ __forceinline__ uint32_t ld_cached(const uint32_t* p) { return __ldca(p); }

// Priority coarsening (Section 2): bucket = floor(priority / Delta); A* priority is g + h.
__device__ __forceinline__ uint32_t bucket_of(uint32_t d, uint32_t h, uint32_t delta) {
  if (h == 0) return d / delta;
  return (uint32_t)(((unsigned long long)d + h) / delta);
}

// Warp-uniform reads for control decisions: lane 0 reads, every lane gets its value, so a
// value that changes concurrently can never split the warp between two paths.
__device__ __forceinline__ uint64_t warp_now() {
  uint64_t t = 0;
  if ((threadIdx.x & 31) == 0) t = gtimer();
  return __shfl_sync(FULL, t, 0);
}
__device__ __forceinline__ uint32_t warp_ld(const uint32_t* p) {
  uint32_t v = 0;
  if ((threadIdx.x & 31) == 0) v = ld_relaxed(p);
  return __shfl_sync(FULL, v, 0);
}

// Records the first failed internal bounds check; the caller skips the access.
__device__ __forceinline__ void report_bad(Sync* sy, uint32_t code, uint32_t val, uint32_t aux) {
  if (atomicCAS(&sy->bad_code, 0u, code) == 0u) {
    sy->bad_val = val;
    sy->bad_aux = aux;
  }
  atomicOr(&sy->err, kErrBounds);
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

}  // namespace og
