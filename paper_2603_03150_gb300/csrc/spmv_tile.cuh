// Tiled CSR SpMV core shared by every kernel that multiplies by A~ or A~^T.
//
// A tile is a run of whole rows holding at most BLOCK*E - 4 nonzeros, or one
// chunk of a row too long for a tile ("split row").  Per tile:
//  (1) thread t loads the E consecutive nonzeros of the window
//      [a + tE, a + tE + E), a = the tile start rounded down to 16 bytes,
//      with 128-bit loads of column indices and values, and issues all E
//      gathers v[col] back to back (products stay in registers);
//  (2) the thread walks the row boundaries inside its window: rows that end
//      there are finished at once, the first one with a carry-in if it began
//      in an earlier window, and the row still open at the window's end is
//      carried out;
//  (3) carries are combined by a segmented scan over threads (warp shuffles,
//      then across warps in shared memory), so every thread does the same
//      amount of work whatever the row lengths;
//  (4) finished row sums are staged in shared memory and the epilogue runs
//      as one coalesced loop over the tile's rows.
// A split row's chunks each reduce to one partial sum written to a slot; the
// chunk that arrives last (atomic ticket) adds the slots in chunk order and
// runs the row epilogue, so the sum order is fixed.
#pragma once
#include "common.cuh"

namespace pdhg {

template <typename T, int NV>
struct Gather {
  const T* v[NV];
};

// Nonzeros a tile may hold when each of BLOCK threads owns E of them: the
// window starts up to 3 places before the tile's first nonzero.
__host__ __device__ constexpr int tile_capacity(int block, int e) { return block * e - 4; }

// Rows a tile may hold (bounds the staged row sums in shared memory).
__host__ __device__ constexpr int tile_max_rows(int block) { return block * 4; }

// Shared memory bytes needed by run_tiles for a schedule.
template <typename T, int NV, int BLOCK>
__host__ __device__ constexpr size_t tile_smem_bytes(int max_rows) {
  return sizeof(int32_t) * (size_t)(max_rows + 4)   // row offsets of the tile
         + sizeof(T) * (size_t)NV * (max_rows + 4)  // staged row sums
         + sizeof(int32_t) * 2 * (BLOCK / 32)       // first/last key per warp
         + sizeof(T) * (size_t)NV * (BLOCK / 32)    // last value per warp
         + 64;
}

// Epilogue concept:  __device__ void row(int r, const T (&s)[NV], int split_group)
// split_group < 0 for rows completed inside one tile; otherwise the index of
// the split group whose last chunk is finishing the row.
// Optional, called by every thread of the block:
//   __device__ bool begin_tile(const Tile&)   false skips the tile
//   __device__ void end_tile(const Tile&, int tile_index)
template <class Epi>
__device__ __forceinline__ auto epi_begin(Epi& e, const Tile& t, int) -> decltype(e.begin_tile(t)) {
  return e.begin_tile(t);
}
template <class Epi>
__device__ __forceinline__ bool epi_begin(Epi&, const Tile&, long) {
  return true;
}
template <class Epi>
__device__ __forceinline__ auto epi_end(Epi& e, const Tile& t, int i, int) -> decltype(e.end_tile(t, i)) {
  e.end_tile(t, i);
}
template <class Epi>
__device__ __forceinline__ void epi_end(Epi&, const Tile&, int, long) {}
template <typename T, int NV, int BLOCK, int E, class Epi>
__device__ __forceinline__ void run_tiles(const SchedView& S, const int32_t* __restrict__ row_ptr,
                                          const int32_t* __restrict__ col,
                                          const T* __restrict__ val, const Gather<T, NV>& g,
                                          Epi& epi, unsigned char* smem) {
  static_assert(E % 4 == 0, "E must be a multiple of 4");
  constexpr int NW = BLOCK / 32;
  const int rstride = S.max_rows + 4;
  int32_t* rps = reinterpret_cast<int32_t*>(smem);
  int32_t* wfirst = rps + rstride;
  int32_t* wlast = wfirst + NW;
  T* rsum = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(wlast + NW) + 15) & ~uintptr_t(15));
  T* wsum = rsum + NV * rstride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
    const Tile tl = S.tiles[t];
    if (!epi_begin(epi, tl, 0)) continue;
    const int nzb = tl.nz_begin, nze = tl.nz_end;
    const int w0 = (nzb & ~3) + tid * E;

    // (1) loads and gathers
    int cidx[E];
    T vv[E];
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
      const int k4 = w0 + 4 * q;
      if (k4 < nze) {
        const int4 c4 = ldg_int4(col + k4);
        Vec4<T> v4;
        v4.load(val + k4);
        cidx[4 * q + 0] = c4.x;
        cidx[4 * q + 1] = c4.y;
        cidx[4 * q + 2] = c4.z;
        cidx[4 * q + 3] = c4.w;
#pragma unroll
        for (int e = 0; e < 4; ++e) vv[4 * q + e] = v4.v[e];
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          cidx[4 * q + e] = 0;
          vv[4 * q + e] = T(0);
        }
      }
    }
    T p[NV][E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = w0 + e;
      const bool in = k >= nzb && k < nze;
#pragma unroll
      for (int v = 0; v < NV; ++v) p[v][e] = in ? vv[e] * __ldg(g.v[v] + cidx[e]) : T(0);
    }

    if (tl.split >= 0) {
      // one chunk of a long row: block sum, then the ordered slot combine
      T s[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        s[v] = T(0);
#pragma unroll
        for (int e = 0; e < E; ++e) s[v] += p[v][e];
        s[v] = warp_sum(s[v]);
        if (lane == 0) wsum[v * NW + warp] = s[v];
      }
      __syncthreads();
      if (tid == 0) {
        T part[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          part[v] = T(0);
          for (int w = 0; w < NW; ++w) part[v] += wsum[v * NW + w];
        }
        T* slots = reinterpret_cast<T*>(S.slots);
        const SplitGroup grp = S.groups[tl.split];
#pragma unroll
        for (int v = 0; v < NV; ++v) slots[(size_t)(grp.slot0 + tl.part) * NV + v] = part[v];
        __threadfence();
        const int prev = atomicAdd(S.counters + tl.split, 1);
        if (prev == grp.nparts - 1) {
          __threadfence();
          T tot[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) tot[v] = T(0);
          for (int pp = 0; pp < grp.nparts; ++pp)
#pragma unroll
            for (int v = 0; v < NV; ++v) tot[v] += __ldcg(slots + (size_t)(grp.slot0 + pp) * NV + v);
          S.counters[tl.split] = 0;
          epi.row(grp.row, tot, tl.split);
        }
      }
      __syncthreads();
      epi_end(epi, tl, t, 0);
      continue;
    }

    // row offsets of the tile (absolute nonzero positions)
    const int nrows = tl.row_end - tl.row_begin;
    for (int r = tid; r <= nrows; r += BLOCK) rps[r] = __ldg(row_ptr + tl.row_begin + r);
    __syncthreads();

    // (2) walk the row ends inside this thread's window
    const int k0 = max(w0, nzb), k1 = min(w0 + E, nze);
    int key = -1, head_row = -1;
    T acc[NV], head_val[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = head_val[v] = T(0);
    if (k0 < k1) {
      // row holding k0: the last r with rps[r] <= k0 (skips empty rows)
      int lo = 0, hi = nrows;  // invariant: rps[lo] <= k0 < rps[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rps[mid] <= k0) lo = mid; else hi = mid;
      }
      int r = lo;
      int next_end = rps[r + 1];
      bool open = false, first = true;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = w0 + e;
        if (k >= k0 && k < k1) {
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v] += p[v][e];
          open = true;
          if (k + 1 == next_end) {
            if (first && rps[r] < k0) {
              head_row = r;
#pragma unroll
              for (int v = 0; v < NV; ++v) head_val[v] = acc[v];
            } else {
#pragma unroll
              for (int v = 0; v < NV; ++v) rsum[v * rstride + r] = acc[v];
            }
            first = false;
            open = false;
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] = T(0);
            ++r;
            while (r < nrows && rps[r + 1] == rps[r]) ++r;
            next_end = (r < nrows) ? rps[r + 1] : 0x7fffffff;
          }
        }
      }
      if (open) key = r;
    }

    // (3) segmented inclusive scan of the open carries over threads
    T sv[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) sv[v] = (key >= 0) ? acc[v] : T(0);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int ko = __shfl_up_sync(0xffffffffu, key, off);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T o = __shfl_up_sync(0xffffffffu, sv[v], off);
        if (lane >= off && ko == key) sv[v] += o;
      }
    }
    const unsigned same = __match_any_sync(0xffffffffu, key);
    if (lane == 31) {
      wlast[warp] = key;
#pragma unroll
      for (int v = 0; v < NV; ++v) wsum[v * NW + warp] = sv[v];
    }
    if (lane == 0) wfirst[warp] = key;
    __syncthreads();
    if (key >= 0 && (same & 1u)) {  // this run reaches back to lane 0
      for (int w = warp - 1; w >= 0; --w) {
        if (wlast[w] != key) break;
#pragma unroll
        for (int v = 0; v < NV; ++v) sv[v] += wsum[v * NW + w];
        if (wfirst[w] != key) break;
      }
    }
    // carry-in of a row that began before this window: the previous thread's
    // scan value when it carries the same row (from the previous warp for lane 0)
    const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
    T cprev[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) cprev[v] = __shfl_up_sync(0xffffffffu, sv[v], 1);
    if (head_row >= 0) {
      if (lane > 0) {
        if (kprev == head_row)
#pragma unroll
          for (int v = 0; v < NV; ++v) head_val[v] += cprev[v];
      } else {
        for (int w = warp - 1; w >= 0; --w) {
          if (wlast[w] != head_row) break;
#pragma unroll
          for (int v = 0; v < NV; ++v) head_val[v] += wsum[v * NW + w];
          if (wfirst[w] != head_row) break;
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) rsum[v * rstride + head_row] = head_val[v];
    }
    __syncthreads();

    // (4) epilogue, one coalesced pass over the tile's rows
    for (int r = tid; r < nrows; r += BLOCK) {
      T s[NV];
      const bool empty = rps[r] == rps[r + 1];
#pragma unroll
      for (int v = 0; v < NV; ++v) s[v] = empty ? T(0) : rsum[v * rstride + r];
      epi.row(tl.row_begin + r, s, -1);
    }
    __syncthreads();
    epi_end(epi, tl, t, 0);
  }
}

// ---------------------------------------------------------------------------
// Vector variant for matrices whose rows are all short: G consecutive lanes
// own one row, read its nonzeros with a G-strided loop straight from global
// memory, gather, and reduce with shuffles; the row sums are staged in shared
// memory and the epilogue runs as one coalesced loop over the tile's rows
// (two block barriers per tile, no row search or carry scan).  Split tiles
// reduce over the whole block as above.
// ---------------------------------------------------------------------------
template <typename T, int NV, int BLOCK, int G, class Epi>
__device__ __forceinline__ void run_tiles_vec(const SchedView& S, const int32_t* __restrict__ row_ptr,
                                              const int32_t* __restrict__ col,
                                              const T* __restrict__ val, const Gather<T, NV>& g,
                                              Epi& epi, unsigned char* smem) {
  static_assert(G >= 1 && G <= 32 && (G & (G - 1)) == 0, "G must be a power of two <= 32");
  constexpr int NW = BLOCK / 32;
  const int rstride = S.max_rows + 4;
  T* rsum = reinterpret_cast<T*>(smem);
  T* wsum = rsum + NV * rstride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = tid / G, gl = tid & (G - 1);
  constexpr int NG = BLOCK / G;
  for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
    const Tile tl = S.tiles[t];
    if (!epi_begin(epi, tl, 0)) continue;
    if (tl.split >= 0) {
      T s[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) s[v] = T(0);
      for (int k = tl.nz_begin + tid; k < tl.nz_end; k += BLOCK) {
        const T a = __ldg(val + k);
        const int c = __ldg(col + k);
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] += a * __ldg(g.v[v] + c);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        s[v] = warp_sum(s[v]);
        if (lane == 0) wsum[v * NW + warp] = s[v];
      }
      __syncthreads();
      if (tid == 0) {
        T part[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          part[v] = T(0);
          for (int w = 0; w < NW; ++w) part[v] += wsum[v * NW + w];
        }
        T* slots = reinterpret_cast<T*>(S.slots);
        const SplitGroup sg = S.groups[tl.split];
#pragma unroll
        for (int v = 0; v < NV; ++v) slots[(size_t)(sg.slot0 + tl.part) * NV + v] = part[v];
        __threadfence();
        const int prev = atomicAdd(S.counters + tl.split, 1);
        if (prev == sg.nparts - 1) {
          __threadfence();
          T tot[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) tot[v] = T(0);
          for (int pp = 0; pp < sg.nparts; ++pp)
#pragma unroll
            for (int v = 0; v < NV; ++v) tot[v] += __ldcg(slots + (size_t)(sg.slot0 + pp) * NV + v);
          S.counters[tl.split] = 0;
          epi.row(sg.row, tot, tl.split);
        }
      }
      __syncthreads();
      epi_end(epi, tl, t, 0);
      continue;
    }
    const int nrows = tl.row_end - tl.row_begin;
    // every lane walks the same number of group rounds (shuffles need all 32)
    for (int r0 = 0; r0 < nrows; r0 += NG) {
      const int r = tl.row_begin + r0 + grp;
      T s[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) s[v] = T(0);
      if (r0 + grp < nrows) {
        const int e = __ldg(row_ptr + r + 1);
        for (int k = __ldg(row_ptr + r) + gl; k < e; k += G) {
          const T a = __ldg(val + k);
          const int c = __ldg(col + k);
#pragma unroll
          for (int v = 0; v < NV; ++v) s[v] += a * __ldg(g.v[v] + c);
        }
      }
#pragma unroll
      for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] += __shfl_down_sync(0xffffffffu, s[v], o, G);
      if (gl == 0 && r0 + grp < nrows)
#pragma unroll
        for (int v = 0; v < NV; ++v) rsum[v * rstride + r0 + grp] = s[v];
    }
    __syncthreads();
    for (int r = tid; r < nrows; r += BLOCK) {
      T s[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) s[v] = rsum[v * rstride + r];
      epi.row(tl.row_begin + r, s, -1);
    }
    __syncthreads();
    epi_end(epi, tl, t, 0);
  }
}

// Schedule variant V: V > 0 segmented with E = V nonzeros per thread,
// V < 0 vector with G = -V lanes per row.
template <typename T, int NV, int BLOCK, int V, class Epi>
__device__ __forceinline__ void run_sched(const SchedView& S, const int32_t* __restrict__ row_ptr,
                                          const int32_t* __restrict__ col,
                                          const T* __restrict__ val, const Gather<T, NV>& g,
                                          Epi& epi, unsigned char* smem) {
  if constexpr (V > 0)
    run_tiles<T, NV, BLOCK, V>(S, row_ptr, col, val, g, epi, smem);
  else
    run_tiles_vec<T, NV, BLOCK, -V>(S, row_ptr, col, val, g, epi, smem);
}

// Shared memory of run_tiles_vec (staged row sums, split-tile block sums).
template <typename T, int NV, int BLOCK>
__host__ __device__ constexpr size_t tile_vec_smem_bytes(int max_rows) {
  return sizeof(T) * (size_t)NV * (max_rows + 4) + sizeof(T) * (size_t)NV * (BLOCK / 32) + 16;
}

}  // namespace pdhg
