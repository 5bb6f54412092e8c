// Vertex order on the device: the hot-first packing of a skewed graph.
//
// The searches read dist[v] at random for every relaxed edge, and on a power-law graph
// most of those reads go to a small set of high-degree vertices.  With the user's
// numbering those vertices are spread over the whole distance array, so every cache line
// of it is partly hot; moving them to ids [0, K) in order of degree packs the hot words
// into K / 8 sectors per query that stay in L2 (the hottest at the front, where L1 keeps
// some).  Only the moved vertices change id, so a per-vertex array goes from one order
// to the other by a gather and a scatter over the moved list.
#include <cuda_runtime.h>
#include <stdint.h>

namespace og {

// New adjacency in the new order: vertex x takes the row of vertex src_of[x] (an id of
// the current order), each neighbour id mapped through new_of (current -> new).  One
// warp per vertex, lanes over the row.
__global__ void og_pack_adj_kernel(const uint32_t* off_old, const uint2* adj_old,
                                   const uint32_t* off_new, const uint32_t* src_of,
                                   const uint32_t* new_of, uint2* adj_new, uint32_t n) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t x = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += nwarps) {
    const uint32_t u = src_of[x];
    const uint32_t beg = off_old[u], deg = off_old[u + 1] - beg;
    const uint32_t dst = off_new[x];
    for (uint32_t i = lane; i < deg; i += 32) {
      uint2 e = adj_old[beg + i];
      e.x = new_of[e.x];
      adj_new[dst + i] = e;
    }
  }
}

// Moved list mv[i] = {device id, user id} of the i-th moved vertex.  Gather: tmp[r][i] =
// rows[r][from(i)]; scatter: rows[r][to(i)] = tmp[r][i], with (from, to) = (device, user)
// for rows in the device order going to the user's, (user, device) the other way.  The
// moved device ids and user ids are the same set, so the two passes permute in place.
__global__ void og_perm_gather_kernel(const uint32_t* rows, uint32_t n, uint32_t nrows,
                                      const uint2* mv, uint32_t nmv, uint32_t to_user,
                                      uint32_t* tmp) {
  const size_t total = (size_t)nmv * nrows;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const uint32_t r = (uint32_t)(i / nmv), k = (uint32_t)(i % nmv);
    const uint2 p = mv[k];
    tmp[i] = rows[(size_t)r * n + (to_user ? p.x : p.y)];
  }
}

__global__ void og_perm_scatter_kernel(uint32_t* rows, uint32_t n, uint32_t nrows,
                                       const uint2* mv, uint32_t nmv, uint32_t to_user,
                                       const uint32_t* tmp) {
  const size_t total = (size_t)nmv * nrows;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const uint32_t r = (uint32_t)(i / nmv), k = (uint32_t)(i % nmv);
    const uint2 p = mv[k];
    rows[(size_t)r * n + (to_user ? p.y : p.x)] = tmp[i];
  }
}

cudaError_t launch_pack_adj(const uint32_t* off_old, const uint2* adj_old,
                            const uint32_t* off_new, const uint32_t* src_of,
                            const uint32_t* new_of, uint2* adj_new, uint32_t n, int sms,
                            cudaStream_t st) {
  og_pack_adj_kernel<<<sms * 8, 256, 0, st>>>(off_old, adj_old, off_new, src_of, new_of,
                                              adj_new, n);
  return cudaGetLastError();
}

cudaError_t launch_perm_rows(uint32_t* rows, uint32_t n, uint32_t nrows, const uint2* mv,
                             uint32_t nmv, bool to_user, uint32_t* tmp, int sms,
                             cudaStream_t st) {
  if (nmv == 0 || nrows == 0) return cudaSuccess;
  og_perm_gather_kernel<<<sms * 8, 256, 0, st>>>(rows, n, nrows, mv, nmv, to_user ? 1u : 0u,
                                                 tmp);
  og_perm_scatter_kernel<<<sms * 8, 256, 0, st>>>(rows, n, nrows, mv, nmv, to_user ? 1u : 0u,
                                                  tmp);
  return cudaGetLastError();
}

}  // namespace og
