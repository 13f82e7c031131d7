// Tiled CSR SpMV core shared by every kernel that multiplies by A~ or A~^T.
//
// Per tile: (1) stream the tile's column indices and values with 128-bit
// loads from a 16-byte aligned start (elements outside the tile are masked),
// form val * v[col] for NV gathered vectors, and stage the products in shared
// memory; (2) reduce each row's products with a group of `lanes` threads
// (warp shuffles, plus a shared-memory step when a group spans warps); (3)
// hand the row sums to the caller's epilogue.  Rows longer than the tile are
// split across tiles and combined in a fixed order (see SchedView).
#pragma once
#include "common.cuh"

namespace pdhg {

template <typename T, int NV>
struct Gather {
  const T* v[NV];
};

// Staged products per vector: the tile's nonzeros start up to 3 places
// after the 16-byte aligned load start, and the last 4-wide store may run 3
// past the tile end, so round up to a multiple of 4 with 4 spare.
__host__ __device__ constexpr int prod_stride(int tile_nnz) { return (tile_nnz + 3) / 4 * 4 + 4; }

// Shared memory bytes needed by run_tiles for a schedule.
template <typename T, int NV, int BLOCK>
__host__ __device__ constexpr size_t tile_smem_bytes(int tile_nnz, int max_rows) {
  return sizeof(T) * (size_t)NV * prod_stride(tile_nnz) + sizeof(int32_t) * (size_t)(max_rows + 4) +
         sizeof(T) * (size_t)NV * (BLOCK / 32) + 16;
}

// Epilogue concept:  __device__ void row(int r, const T (&s)[NV], int split_group)
// split_group < 0 for rows completed inside one tile; otherwise the index of
// the split group whose last chunk is finishing the row.
template <typename T, int NV, int BLOCK, class Epi>
__device__ __forceinline__ void run_tiles(const SchedView& S, const int32_t* __restrict__ row_ptr,
                                          const int32_t* __restrict__ col,
                                          const T* __restrict__ val, const Gather<T, NV>& g,
                                          Epi& epi, unsigned char* smem) {
  const int pstride = prod_stride(S.tile_nnz);
  T* prod = reinterpret_cast<T*>(smem);
  int32_t* rp = reinterpret_cast<int32_t*>(prod + NV * pstride);
  T* red = reinterpret_cast<T*>(
      (reinterpret_cast<uintptr_t>(rp + S.max_rows + 4) + 15) & ~uintptr_t(15));

  for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
    const Tile tl = S.tiles[t];
    const int a = tl.nz_begin & ~3;
    // (1) products into shared memory
    for (int k4 = a + 4 * (int)threadIdx.x; k4 < tl.nz_end; k4 += 4 * BLOCK) {
      const int4 c4 = ldg_int4(col + k4);
      Vec4<T> v4;
      v4.load(val + k4);
      const int cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Vec4<T> p;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = k4 + e;
          p.v[e] = (k >= tl.nz_begin && k < tl.nz_end) ? v4.v[e] * __ldg(g.v[v] + cc[e]) : T(0);
        }
        p.store_smem(prod + v * pstride + (k4 - a));
      }
    }
    const int nrows = tl.row_end - tl.row_begin;
    if (tl.split < 0) {
      for (int r = threadIdx.x; r <= nrows; r += BLOCK) rp[r] = __ldg(row_ptr + tl.row_begin + r) - a;
    } else if (threadIdx.x == 0) {
      rp[0] = tl.nz_begin - a;
      rp[1] = tl.nz_end - a;
    }
    __syncthreads();

    // (2) row reductions
    const int G = tl.lanes;
    auto finish = [&](int r, T (&s)[NV]) {
      if (tl.split < 0) {
        epi.row(tl.row_begin + r, s, -1);
        return;
      }
      T* slots = reinterpret_cast<T*>(S.slots);
      const SplitGroup grp = S.groups[tl.split];
#pragma unroll
      for (int v = 0; v < NV; ++v) slots[(size_t)(grp.slot0 + tl.part) * NV + v] = s[v];
      __threadfence();
      const int prev = atomicAdd(S.counters + tl.split, 1);
      if (prev == grp.nparts - 1) {
        __threadfence();
        T tot[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) tot[v] = T(0);
        for (int p = 0; p < grp.nparts; ++p)
#pragma unroll
          for (int v = 0; v < NV; ++v) tot[v] += __ldcg(slots + (size_t)(grp.slot0 + p) * NV + v);
        S.counters[tl.split] = 0;
        epi.row(grp.row, tot, tl.split);
      }
    };

    if (G <= 32) {
      const int groups = BLOCK / G;
      const int gid = threadIdx.x / G, lane = threadIdx.x & (G - 1);
      for (int r0 = 0; r0 < nrows; r0 += groups) {
        const int r = r0 + gid;
        T s[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] = T(0);
        if (r < nrows) {
          const int e = rp[r + 1];
          for (int k = rp[r] + lane; k < e; k += G)
#pragma unroll
            for (int v = 0; v < NV; ++v) s[v] += prod[v * pstride + k];
        }
        for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
          for (int v = 0; v < NV; ++v) s[v] += __shfl_down_sync(0xffffffffu, s[v], o, G);
        if (lane == 0 && r < nrows) finish(r, s);
      }
    } else {
      const int groups = BLOCK / G, wpg = G / 32;
      const int gid = threadIdx.x / G, lane = threadIdx.x % G, warp = threadIdx.x >> 5;
      for (int r0 = 0; r0 < nrows; r0 += groups) {
        const int r = r0 + gid;
        T s[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] = T(0);
        if (r < nrows) {
          const int e = rp[r + 1];
          for (int k = rp[r] + lane; k < e; k += G)
#pragma unroll
            for (int v = 0; v < NV; ++v) s[v] += prod[v * pstride + k];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          s[v] = warp_sum(s[v]);
          if ((threadIdx.x & 31) == 0) red[v * (BLOCK / 32) + warp] = s[v];
        }
        __syncthreads();
        if (lane == 0 && r < nrows) {
          T tot[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            tot[v] = T(0);
            for (int w = 0; w < wpg; ++w) tot[v] += red[v * (BLOCK / 32) + gid * wpg + w];
          }
          finish(r, tot);
        }
        __syncthreads();
      }
    }
    __syncthreads();
  }
}

}  // namespace pdhg
