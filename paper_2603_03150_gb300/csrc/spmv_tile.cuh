// Tiled CSR SpMV core shared by every kernel that multiplies by A~ or A~^T.
//
// A tile is a run of whole rows holding at most BLOCK*E - 4 nonzeros, or one
// chunk of a row too long for a tile ("split row"), or a run of rows without
// nonzeros.  Per tile of whole rows:
//  (1) thread t owns the E consecutive nonzeros of the window
//      [a + tE, a + tE + E), a = the tile start rounded down to 16 bytes; in
//      steps of 8 it loads column indices and values with 128-bit loads
//      (L2 evict-first, no L1 allocation) and issues the 8 gathers v[col]
//      back to back;
//  (2) the thread walks the row ends inside its window with one fused
//      multiply-add per nonzero, the row structure read from a window word
//      computed once with the schedule (row-end mask, first row, "continues
//      a row" bit): rows that end there are finished at once, the first one
//      with a carry-in if it began in an earlier window, and the row still
//      open at the window's end is carried out;
//  (3) carries are combined by a segmented scan over threads (warp shuffles,
//      then across warps in shared memory), so every thread does the same
//      amount of work whatever the row lengths;
//  (4) finished row sums are staged in shared memory and the epilogue runs
//      as one coalesced loop over the tile's rows.
// A split row's chunks each reduce to one partial sum written to a slot; the
// chunk that arrives last (atomic ticket) adds the slots in chunk order and
// runs the row epilogue, so the sum order is fixed.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace pdhg {

// The vectors a tile kernel gathers: load(c, o) gives entry c of each.
template <typename T, int NV>
struct Gather {
  const T* v[NV];
  __device__ __forceinline__ void load(int c, T (&o)[NV]) const {
#pragma unroll
    for (int q = 0; q < NV; ++q) o[q] = __ldg(v[q] + c);
  }
};

// Two vectors stored interleaved (entry c of each at p[2c], p[2c + 1]): one
// 8- or 16-byte load per nonzero instead of two scattered ones.
template <typename T>
struct GatherPair {
  const T* p;
  __device__ __forceinline__ void load(int c, T (&o)[2]) const {
    if constexpr (sizeof(T) == 4) {
      const float2 q = __ldg(reinterpret_cast<const float2*>(p) + c);
      o[0] = q.x;
      o[1] = q.y;
    } else {
      const double2 q = __ldg(reinterpret_cast<const double2*>(p) + c);
      o[0] = q.x;
      o[1] = q.y;
    }
  }
};

// Nonzeros a tile may hold when each of BLOCK threads owns E of them: the
// window starts up to 3 places before the tile's first nonzero.
__host__ __device__ constexpr int tile_capacity(int block, int e) { return block * e - 4; }

// Rows a tile may hold (bounds the staged row sums in shared memory).
__host__ __device__ constexpr int tile_max_rows(int block) { return block * 4; }

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

// One chunk of a split row: block sum of the threads' partial sums (each the
// sum of its window's products in nonzero order), then the ordered slot
// combine (the chunk that arrives last adds the slots in chunk order and runs
// the row epilogue).  Ends with a block barrier.
template <typename T, int NV, int BLOCK, class Epi>
__device__ __forceinline__ void split_chunk(const SchedView& S, const Tile& tl,
                                            const T (&part_in)[NV], Epi& epi, T* wsum) {
  constexpr int NW = BLOCK / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T sv = warp_sum(part_in[v]);
    if (lane == 0) wsum[v * NW + warp] = sv;
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
}

// Combines the open carries of a whole-row tile.  Each thread passes the row
// whose sum is still open at the end of its window (key, -1 if none) with its
// partial sum acc, and the row it closed first if that row began before its
// window (head_row, -1 if none) with the partial sum head_val; the carries of
// equal keys are added by a segmented scan over threads in thread order and
// the head rows are written to rsum.  Ends with a barrier.
template <typename T, int NV, int BLOCK>
__device__ __forceinline__ void carry_combine(int key, const T (&acc)[NV], int head_row,
                                              T (&head_val)[NV], T* rsum, int rstride,
                                              int32_t* wfirst, int32_t* wlast, T* wsum) {
  constexpr int NW = BLOCK / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // segmented inclusive scan of the open carries over threads
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
}

// ---------------------------------------------------------------------------
// Window words.  The row structure of every thread window of a whole-row
// tile is computed once when the schedule is built (one word per window;
// tile.word0 = index of the tile's first word, schedule view .wd).  With
// M = 16 mask bits (32-bit words, E <= 16) or M = 32 (64-bit words, E = 32):
//   bits 0..M-1   row-end mask: bit e set when nonzero w0+e is its row's last
//   bit  M        the window's first nonzero continues a row begun before it
//   bits M+1..    row of the window's first nonzero, relative to row_begin
// Tiles of whole rows hold no row without nonzeros (such rows form tiles of
// their own, nz_begin == nz_end), so the walk is one mask test per nonzero.
// ---------------------------------------------------------------------------
template <int E>
struct WindowWord {
  using type = typename std::conditional<(E > 16), uint64_t, uint32_t>::type;
  static constexpr int kMaskBits = E > 16 ? 32 : 16;
};

template <int E>
__host__ __device__ constexpr typename WindowWord<E>::type window_word(int first_row, bool head,
                                                                       uint64_t mask) {
  using W = typename WindowWord<E>::type;
  return ((W)first_row << (WindowWord<E>::kMaskBits + 1)) |
         ((W)(head ? 1u : 0u) << WindowWord<E>::kMaskBits) | (W)mask;
}

// Segmented tile SpMV (row_ptr is not read: the window words carry the rows).
// A thread's window of E nonzeros is loaded, gathered and walked in steps of
// EC = 8 (E = 16, 32: the per-tile work - descriptor, carry scan, barriers -
// is shared by more nonzeros at the register cost of E = 8).
template <typename T, int NV, int BLOCK, int E, class Epi, class Gv>
__device__ __forceinline__ void run_tiles(const SchedView& S, const int32_t* __restrict__ /*row_ptr*/,
                                          const int32_t* __restrict__ col,
                                          const T* __restrict__ val, const Gv& g,
                                          Epi& epi, unsigned char* smem) {
  static_assert(E % 4 == 0 && E <= 32, "E must be a multiple of 4, at most 32");
  using W = typename WindowWord<E>::type;
  constexpr int MB = WindowWord<E>::kMaskBits;
  constexpr int EC = E < 8 ? E : 8;
  constexpr int NW = BLOCK / 32;
  const int rstride = S.max_rows + 4;
  int32_t* wfirst = reinterpret_cast<int32_t*>(smem);
  int32_t* wlast = wfirst + NW;
  T* rsum = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(wlast + NW) + 15) & ~uintptr_t(15));
  T* wsum = rsum + NV * rstride;
  const int tid = threadIdx.x;
  const W* __restrict__ wd = reinterpret_cast<const W*>(S.wd);
  const uint64_t pol = stream_policy();

  for (int t = blockIdx.x; t < S.ntiles; t += gridDim.x) {
    const Tile tl = S.tiles[t];
    // the block's next tile: its descriptor now, its nonzeros and window
    // words prefetched into L2 once this tile's own loads are out
    const bool has_next = tid == 0 && t + (int)gridDim.x < S.ntiles;
    Tile nx{};
    if (has_next) nx = S.tiles[t + gridDim.x];
    if (!epi_begin(epi, tl, 0)) continue;
    const int nzb = tl.nz_begin, nze = tl.nz_end;
    const int nrows = tl.row_end - tl.row_begin;
    if (nzb == nze) {  // rows without nonzeros: zero sums
      T z[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) z[v] = T(0);
      for (int r = tid; r < nrows; r += BLOCK) epi.row(tl.row_begin + r, z, -1);
      __syncthreads();
      epi_end(epi, tl, t, 0);
      continue;
    }
    const int w0 = (nzb & ~3) + tid * E;
    const W d = tl.split < 0 ? ld_stream(wd + tl.word0 + tid, pol) : W(0);

    // load, gather and walk; nonzeros outside [nzb, nze) add zero and carry
    // no mask bit (split chunks have no mask bits: acc is the window's sum)
    int r = (int)(d >> (MB + 1));
    bool head = (d >> MB) & 1u;
    int head_row = -1;
    T acc[NV], head_val[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = head_val[v] = T(0);
#pragma unroll
    for (int c = 0; c < E / EC; ++c) {
      const int wc = w0 + c * EC;
      if (wc >= nze) break;
      int cidx[EC];
      T vv[EC];
#pragma unroll
      for (int q = 0; q < EC / 4; ++q) {
        const int k4 = wc + 4 * q;
        if (k4 < nze) {
          const int4 c4 = ld_stream_int4(col + k4, pol);
          Vec4<T> v4;
          v4.load_stream(val + k4, pol);
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
      // gathered values, zero outside [nzb, nze): the walk then accumulates
      // with one fused multiply-add per nonzero
      T gv[NV][EC];
#pragma unroll
      for (int e = 0; e < EC; ++e) {
        const int k = wc + e;
        const bool in = k >= nzb && k < nze;
        T q[NV];
        if (in) {
          g.load(cidx[e], q);
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) q[v] = T(0);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) gv[v][e] = q[v];
      }
#pragma unroll
      for (int e = 0; e < EC; ++e) {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = fmadd(vv[e], gv[v][e], acc[v]);
        if ((d >> (c * EC + e)) & 1u) {
          if (head) {
            head_row = r;
#pragma unroll
            for (int v = 0; v < NV; ++v) head_val[v] = acc[v];
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) rsum[v * rstride + r] = acc[v];
          }
          head = false;
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v] = T(0);
          ++r;
        }
      }
    }

    if (has_next) {
      prefetch_l2(col + nx.nz_begin, 4LL * (nx.nz_end - nx.nz_begin));
      prefetch_l2(val + nx.nz_begin, (int64_t)sizeof(T) * (nx.nz_end - nx.nz_begin));
      if (nx.split < 0 && nx.nz_end > nx.nz_begin)
        prefetch_l2(wd + nx.word0, (int64_t)sizeof(W) * BLOCK);
    }
    if (tl.split >= 0) {
      split_chunk<T, NV, BLOCK>(S, tl, acc, epi, wsum);
      epi_end(epi, tl, t, 0);
      continue;
    }

    // the row still open at the window's end is carried out
    const int k0 = max(w0, nzb), k1 = min(w0 + E, nze);
    const int key = (k0 < k1 && !((d >> (k1 - 1 - w0)) & 1u)) ? r : -1;
    carry_combine<T, NV, BLOCK>(key, acc, head_row, head_val, rsum, rstride, wfirst, wlast, wsum);

    for (int rr = tid; rr < nrows; rr += BLOCK) {
      T sr[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) sr[v] = rsum[v * rstride + rr];
      epi.row(tl.row_begin + rr, sr, -1);
    }
    __syncthreads();
    epi_end(epi, tl, t, 0);
  }
}

// Shared memory bytes needed by run_tiles for a schedule.
template <typename T, int NV, int BLOCK>
__host__ __device__ constexpr size_t tile_smem_bytes(int max_rows) {
  return sizeof(int32_t) * 2 * (BLOCK / 32) + 16 + sizeof(T) * (size_t)NV * (max_rows + 4) +
         sizeof(T) * (size_t)NV * (BLOCK / 32) + 16;
}

// ---------------------------------------------------------------------------
// Vector variant for matrices whose rows are all short: G consecutive lanes
// own one row, read its nonzeros with a G-strided loop straight from global
// memory, gather, and reduce with shuffles; the row sums are staged in shared
// memory and the epilogue runs as one coalesced loop over the tile's rows
// (two block barriers per tile, no row search or carry scan).  Split tiles
// reduce over the whole block as above.
// ---------------------------------------------------------------------------
template <typename T, int NV, int BLOCK, int G, class Epi, class Gv>
__device__ __forceinline__ void run_tiles_vec(const SchedView& S, const int32_t* __restrict__ row_ptr,
                                              const int32_t* __restrict__ col,
                                              const T* __restrict__ val, const Gv& g,
                                              Epi& epi, unsigned char* smem) {
  static_assert(G >= 1 && G <= 32 && (G & (G - 1)) == 0, "G must be a power of two <= 32");
  constexpr int NW = BLOCK / 32;
  const int rstride = S.max_rows + 4;
  T* rsum = reinterpret_cast<T*>(smem);
  T* wsum = rsum + NV * rstride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t pol = stream_policy();
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
        const T a = ld_stream(val + k, pol);
        const int c = ld_stream(col + k, pol);
        T q[NV];
        g.load(c, q);
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] += a * q[v];
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
          const T a = ld_stream(val + k, pol);
          const int c = ld_stream(col + k, pol);
          T q[NV];
          g.load(c, q);
#pragma unroll
          for (int v = 0; v < NV; ++v) s[v] += a * q[v];
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
template <typename T, int NV, int BLOCK, int V, class Epi, class Gv>
__device__ __forceinline__ void run_sched(const SchedView& S, const int32_t* __restrict__ row_ptr,
                                          const int32_t* __restrict__ col,
                                          const T* __restrict__ val, const Gv& g,
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
