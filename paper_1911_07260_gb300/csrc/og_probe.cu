// Memory round-trip probe (diagnostic, not part of the search path).
//
// Every thread follows its own chain of dependent accesses through a word array: the
// value read at one position is the next position, so each access waits for the one
// before it and the time per hop is one round trip.  The chain visits L lines of 128
// bytes spread evenly over the array (line j at byte j * spacing, spacing = bytes / L)
// in the cycle j -> (j + stride) mod L with an odd stride of about a quarter of L, so
// every hop lands far from the previous one and a chain visits all L lines before it
// repeats.  L * 128 bytes is the footprint: a small footprint stays in L2, and spreading
// it over a large array (a large spacing) adds address-translation misses without cache
// misses.  Run with one warp the chains see the unloaded latency; run at the persistent
// kernels' occupancy they see the latency under that many requests in flight, which is
// what a fused level of the search waits for on each of its dependent steps.  With
// several chains per thread the same kernel measures how many independent random
// accesses a second the memory system serves (threads x chains / time per hop).
#include <cuda_runtime.h>
#include <stdint.h>

#include "og.h"

namespace og {

// Line j holds the word index of line (j + stride) mod L (L a power of two, stride odd);
// spacing_w = words between lines.
__global__ void og_probe_init_kernel(uint32_t* buf, uint32_t lmask, uint32_t stride,
                                     uint32_t spacing_w) {
  const size_t s = (size_t)gridDim.x * blockDim.x;
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j <= lmask; j += s)
    buf[j * spacing_w] = (uint32_t)(((j + stride) & lmask) * spacing_w);
}

// mode 0: ld.relaxed.gpu (served by L2), 1: atomicMin with the result used (an L2
// atomic round trip; the value written is never smaller, so the array is unchanged),
// 2: non-coherent load through L1 (__ldg).  Each thread follows W independent chains,
// so W accesses of a thread are in flight together.
template <int MODE, int W>
__global__ void og_probe_chain_kernel(uint32_t* buf, uint32_t lmask, uint32_t spacing_w,
                                      uint32_t hops, uint32_t* sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t i[W];
#pragma unroll
  for (int k = 0; k < W; ++k)  // starting points on different lines
    i[k] = (((t * W + k) * 40961u) & lmask) * spacing_w;
  for (uint32_t h = 0; h < hops; ++h) {
#pragma unroll
    for (int k = 0; k < W; ++k) {
      if (MODE == 0) {
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(i[k]) : "l"(buf + i[k]) : "memory");
      } else if (MODE == 1) {
        i[k] = atomicMin(buf + i[k], 0xFFFFFFFFu);
      } else {
        i[k] = __ldg(buf + i[k]);
      }
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) x |= i[k];
  if (x == 0xFFFFFFFFu) *sink = t;  // never true: keeps the chains live
}

template <int MODE>
void launch_probe(uint32_t chains, uint32_t ctas, uint32_t threads, uint32_t* buf,
                  uint32_t lmask, uint32_t spacing_w, uint32_t hops, uint32_t* sink) {
  switch (chains) {
    case 1: og_probe_chain_kernel<MODE, 1><<<ctas, threads>>>(buf, lmask, spacing_w, hops, sink); break;
    case 2: og_probe_chain_kernel<MODE, 2><<<ctas, threads>>>(buf, lmask, spacing_w, hops, sink); break;
    case 4: og_probe_chain_kernel<MODE, 4><<<ctas, threads>>>(buf, lmask, spacing_w, hops, sink); break;
    case 8: og_probe_chain_kernel<MODE, 8><<<ctas, threads>>>(buf, lmask, spacing_w, hops, sink); break;
    default: og_probe_chain_kernel<MODE, 16><<<ctas, threads>>>(buf, lmask, spacing_w, hops, sink); break;
  }
}

}  // namespace og

extern "C" int og_probe_chain(uint32_t mode, uint64_t bytes, uint64_t footprint,
                              uint32_t ctas, uint32_t threads, uint32_t chains,
                              uint32_t hops, double* ns_per_hop) {
  using namespace og;
  if (!ns_per_hop || mode > 2 || bytes < 4096 || (bytes & (bytes - 1)) || bytes > (16ull << 30) ||
      footprint < 4096 || (footprint & (footprint - 1)) || footprint > bytes || ctas == 0 ||
      threads == 0 || threads > 1024 || threads % 32 || hops == 0 ||
      (chains != 1 && chains != 2 && chains != 4 && chains != 8 && chains != 16))
    return OG_E_INVALID;
  const uint64_t words = bytes / 4;
  const uint64_t lines = footprint / 128;
  const uint32_t lmask = (uint32_t)(lines - 1);
  const uint32_t spacing_w = (uint32_t)(words / lines);             // >= 32 words
  const uint32_t stride = (uint32_t)(((lines / 4) | 1u) + 2u * 7u) & lmask;  // odd, ~L/4
  uint32_t* buf = nullptr;
  uint32_t* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = OG_OK;
  float ms = 0.f;
  auto launch = [&](uint32_t h) {
    if (mode == 0) launch_probe<0>(chains, ctas, threads, buf, lmask, spacing_w, h, sink);
    else if (mode == 1) launch_probe<1>(chains, ctas, threads, buf, lmask, spacing_w, h, sink);
    else launch_probe<2>(chains, ctas, threads, buf, lmask, spacing_w, h, sink);
  };
  if (cudaMalloc(&buf, words * 4) != cudaSuccess || cudaMalloc(&sink, 4) != cudaSuccess) {
    rc = OG_E_OOM;
    goto done;
  }
  if (cudaMemsetAsync(buf, 0, words * 4) != cudaSuccess) {
    rc = OG_E_CUDA;
    goto done;
  }
  og_probe_init_kernel<<<1024, 256>>>(buf, lmask, stride, spacing_w);
  launch(hops < 64 ? hops : 64);  // warm-up (instruction cache, TLB)
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = OG_E_CUDA;
    goto done;
  }
  cudaEventRecord(e0);
  launch(hops);
  cudaEventRecord(e1);
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
    rc = OG_E_CUDA;
    goto done;
  }
  *ns_per_hop = (double)ms * 1.0e6 / (double)hops;
done:
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  return rc;
}
