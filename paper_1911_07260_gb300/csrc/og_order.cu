// Vertex order on the device: the hot-first packing of a skewed graph.
//
// The searches read dist[v] at random for every relaxed edge, and on a power-law graph
// most of those reads go to a small set of high-degree vertices.  With the user's
// numbering those vertices are spread over the whole distance array, so every cache line
// of it is partly hot; moving them to ids [0, K) packs the hot words into K / 8 sectors
// per query that stay in L2.  The packing is a set of disjoint transpositions (a, b) of
// vertex ids (an involution pi), so the same pair list maps a per-vertex array from the
// device order to the user's and back, touching only the moved entries.
#include <cuda_runtime.h>
#include <stdint.h>

namespace og {

// New adjacency in the permuted order: vertex x takes the row of vertex pi[x], each
// neighbour id mapped through pi.  One warp per vertex, lanes over the row.
__global__ void og_pack_adj_kernel(const uint32_t* off_old, const uint2* adj_old,
                                   const uint32_t* off_new, const uint32_t* pi, uint2* adj_new,
                                   uint32_t n) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t x = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += nwarps) {
    const uint32_t u = pi[x];
    const uint32_t beg = off_old[u], deg = off_old[u + 1] - beg;
    const uint32_t dst = off_new[x];
    for (uint32_t i = lane; i < deg; i += 32) {
      uint2 e = adj_old[beg + i];
      e.x = pi[e.x];
      adj_new[dst + i] = e;
    }
  }
}

// Applies the transpositions to nrows rows of n words: rows[r][a] <-> rows[r][b].
__global__ void og_swap_rows_kernel(uint32_t* rows, uint32_t n, uint32_t nrows,
                                    const uint2* swaps, uint32_t nswap) {
  const size_t total = (size_t)nswap * nrows;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const uint32_t r = (uint32_t)(i / nswap);
    const uint2 p = swaps[i % nswap];
    uint32_t* row = rows + (size_t)r * n;
    const uint32_t t = row[p.x];
    row[p.x] = row[p.y];
    row[p.y] = t;
  }
}

cudaError_t launch_pack_adj(const uint32_t* off_old, const uint2* adj_old,
                            const uint32_t* off_new, const uint32_t* pi, uint2* adj_new,
                            uint32_t n, int sms, cudaStream_t st) {
  og_pack_adj_kernel<<<sms * 8, 256, 0, st>>>(off_old, adj_old, off_new, pi, adj_new, n);
  return cudaGetLastError();
}

cudaError_t launch_swap_rows(uint32_t* rows, uint32_t n, uint32_t nrows, const uint2* swaps,
                             uint32_t nswap, int sms, cudaStream_t st) {
  if (nswap == 0 || nrows == 0) return cudaSuccess;
  og_swap_rows_kernel<<<sms * 8, 256, 0, st>>>(rows, n, nrows, swaps, nswap);
  return cudaGetLastError();
}

}  // namespace og
