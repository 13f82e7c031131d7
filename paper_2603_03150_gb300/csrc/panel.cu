// Column-panel SpMV for the float32 half-steps (the products A~^T y of the
// primal step and A~ x+ of the dual step, Section 2's PDHG iteration).
//
// The gathered vector is staged in shared memory one panel of columns at a
// time, so each random read of x or y is a shared-memory load instead of an
// L1/L2 request.  A half-step is two kernels: k_panel_spmv writes one partial
// sum per (panel, row) pseudo-row, then a row pass adds a row's partials in
// panel order and applies the same row epilogue as the fused CSR kernels.
//
// Layout (see PanelTile in common.cuh): per nonzero a float value and the
// 16-bit column within its panel; per 8 nonzeros a window word
//   bits 0..7   pseudo-row ends (bit e: nonzero 8w+e ends its pseudo-row)
//   bit  16     the window's first nonzero continues a pseudo-row begun before
//   bits 17..   pseudo-row of the window's first nonzero, relative to the tile
// per pseudo-row its row.  A warp owns a tile: lane l holds nonzeros
// [8l, 8l+8), walks its row ends with one fused multiply-add per nonzero and a
// store at each row end, and a segmented shuffle scan joins pseudo-rows that
// cross lanes.  No block
// barrier follows the panel load, so 32 warps per SM run independently.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "context.h"
#include "dispatch.cuh"
#include "epilogues.cuh"
#include "kernels.h"

namespace pdhg {

namespace {

constexpr int kPanelThreads = kPanelWarps * 32;

struct PanelLoad {
  PanelTile tl;
  uint32_t d;
  int4 cc;  // 8 column indices, 16 bits each
  Vec4<float> a0, a1;
};

__device__ __forceinline__ void panel_load(PanelLoad& L, const PanelView& V, const PanelTile* dc,
                                           int t0, int t, int lane, uint64_t pol) {
  L.tl = t - t0 < kPanelDescCache ? dc[t - t0] : V.tiles[t];
  L.d = 0u;
  L.cc = make_int4(0, 0, 0, 0);
#pragma unroll
  for (int e = 0; e < 4; ++e) L.a0.v[e] = L.a1.v[e] = 0.f;
  if (L.tl.nps >= 0 && lane * 8 < L.tl.nz_len) {
    const int base = L.tl.nz_begin + lane * 8;
    L.d = ld_stream(V.wd + (base >> 3), pol);
    L.cc = ld_stream_int4(reinterpret_cast<const int32_t*>(V.col + base), pol);
    L.a0.load_stream(V.val + base, pol);
    L.a1.load_stream(V.val + base + 4, pol);
  }
}

__device__ __forceinline__ int col16(const int4& cc, int e) {
  const uint32_t w = (uint32_t)((e >> 1) == 0 ? cc.x : (e >> 1) == 1 ? cc.y : (e >> 1) == 2 ? cc.z : cc.w);
  return (int)((w >> ((e & 1) * 16)) & 0xffffu);
}

}  // namespace

// partial[p][i] = sum of the pseudo-row (p, i); v is the gathered vector
__global__ void __launch_bounds__(kPanelThreads, 1)
    k_panel_spmv(PanelView V, const float* __restrict__ v, const Scalars* __restrict__ sc) {
  extern __shared__ __align__(16) float smem[];
  const int stage_len = kPanelWarps * V.pscap;
  float* stage = smem;               // [warps][pscap] pseudo-row sums
  PanelTile* dc = reinterpret_cast<PanelTile*>(smem + stage_len);  // the first tiles of the block
  int* next_tile = reinterpret_cast<int*>(smem + stage_len + 4 * kPanelDescCache);
  // the panel load's transaction barrier, in static shared memory: placed in
  // the dynamic region beside the tile counter and the panel, the same
  // kernel took about 1 us longer per launch on the power-law LP
  __shared__ __align__(8) unsigned long long panel_bar;
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&panel_bar);
  float* vs = smem + stage_len + 4 * kPanelDescCache + 4;           // the panel of v
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const PanelBlock bd = V.blocks[blockIdx.x];
  const uint64_t pol = stream_policy();
  // the layout is constant, so everything up to pdl_enter() may overlap the
  // kernel that produces v.  The block's tiles are contiguous: one thread
  // hands their nonzeros, window
  // words and rows to the bulk-copy engine as L2 prefetches (16 KB pieces,
  // the four arrays interleaved in the order the warps consume them)
  if (tid == 0) {
    const PanelTile t0 = V.tiles[bd.t_begin], t1 = V.tiles[bd.t_end - 1];
    const int z0 = t0.nz_begin, z1 = t1.nz_begin + t1.nz_len;
    const int p0 = t0.ps_begin, p1 = t1.ps_begin + (t1.nps < 0 ? 1 : t1.nps);
    uintptr_t lo[4] = {reinterpret_cast<uintptr_t>(V.val + z0), reinterpret_cast<uintptr_t>(V.col + z0),
                       reinterpret_cast<uintptr_t>(V.wd + (z0 >> 3)),
                       reinterpret_cast<uintptr_t>(V.psrow + p0)};
    uintptr_t hi[4] = {reinterpret_cast<uintptr_t>(V.val + z1), reinterpret_cast<uintptr_t>(V.col + z1),
                       reinterpret_cast<uintptr_t>(V.wd + (z1 >> 3)),
                       reinterpret_cast<uintptr_t>(V.psrow + p1)};
    // 16-byte boundaries (the arrays are allocated with 64 bytes to spare)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      lo[a] &= ~uintptr_t(15);
      hi[a] = (hi[a] + 15) & ~uintptr_t(15);
    }
    constexpr uintptr_t kPiece = 16384;
    bool more = true;
    for (uintptr_t off = 0; more; off += kPiece) {
      more = false;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        if (lo[a] + off < hi[a]) {
          const uint32_t sz = (uint32_t)min(hi[a] - (lo[a] + off), kPiece);
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo[a] + off), "r"(sz)
                       : "memory");
          more = true;
        }
      }
    }
  }
  for (int q = tid; q < min(bd.t_end - bd.t_begin, kPanelDescCache); q += kPanelThreads)
    dc[q] = V.tiles[bd.t_begin + q];
  // the first tile of each warp is fixed; the others go to whichever warp
  // finishes first (tile sizes and long pseudo-rows vary)
  if (tid == 0) {
    *next_tile = bd.t_begin + kPanelWarps;
    mbar_init(mb);
  }
  __syncthreads();
  int t = bd.t_begin + warp;
  PanelLoad cur;  // the first tile's loads go out before the wait
  if (t < bd.t_end) panel_load(cur, V, dc, bd.t_begin, t, lane, pol);
  pdl_enter();
  {
    // the panel of v: whole 16-byte pieces by the bulk-copy engine (one
    // thread issues 32 KB copies onto the transaction barrier), the tail by
    // the threads.  The panel starts 32-byte aligned (P is a multiple of 8)
    // and so does its place in shared memory.  The wait is bounded
    // (options.wait_limit_ms): past it the block flags the error, waits once
    // more for its copies in flight, and returns without its work (the solve
    // reports a timeout).  Whether the solve has finished is read while the
    // copies run; a finished solve returns once they have landed (no block
    // exits with a copy into its shared memory in flight).
    const int c0 = bd.panel * V.P;
    const int cnt = min(V.P, V.cols - c0);
    const uint32_t bytes = ((uint32_t)cnt * 4u) & ~15u;
    if (tid == 0) {
      mbar_arrive_expect(mb, bytes + V.tx_extra);
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(vs);
      const char* src = reinterpret_cast<const char*>(v + c0);
      constexpr uint32_t kPiece = 32768;
      for (uint32_t o = 0; o < bytes; o += kPiece) bulk_copy_g2s(dst + o, src + o, min(kPiece, bytes - o), mb);
    }
    const int done = sc->done;  // not written while this kernel runs: the same in every thread
    for (int q = (int)(bytes >> 2) + tid; q < cnt; q += kPanelThreads) vs[q] = __ldg(v + c0 + q);
    const bool ok = mbar_wait(mb, 0, V.wait_ns);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(V.err, 1);
      mbar_wait(mb, 0, V.wait_ns);
      return;
    }
    if (done) return;
  }
  float* st = stage + warp * V.pscap;
  float* part = V.partial + (size_t)bd.panel * V.pstride;
  while (t < bd.t_end) {
    const PanelTile tl = cur.tl;
    int t_next = -1;  // set once the next tile's loads are issued
    if (tl.nps < 0) {  // one long pseudo-row: lanes stride over it, then a warp sum
      float acc = 0.f;
      for (int base = tl.nz_begin + lane * 8; base < tl.nz_begin + tl.nz_len; base += 8 * 32) {
        const int4 cc = ld_stream_int4(reinterpret_cast<const int32_t*>(V.col + base), pol);
        Vec4<float> a0, a1;
        a0.load_stream(V.val + base, pol);
        a1.load_stream(V.val + base + 4, pol);
#pragma unroll
        for (int e = 0; e < 4; ++e) acc = fmaf(a0.v[e], vs[col16(cc, e)], acc);
#pragma unroll
        for (int e = 0; e < 4; ++e) acc = fmaf(a1.v[e], vs[col16(cc, 4 + e)], acc);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) part[ld_stream(V.psrow + tl.ps_begin, pol)] = acc;
    } else {
      // rows of this tile's pseudo-rows (at most 8 per lane), loaded before
      // the gathers; slots past the tile's pseudo-rows are skipped warp-wide
      const int nps = tl.nps;
      int rid[kPanelPsCap / 32];
#pragma unroll
      for (int j = 0; j < kPanelPsCap / 32; ++j) {
        rid[j] = 0;
        if (32 * j < nps) {
          const int k = lane + 32 * j;
          if (k < nps) rid[j] = ld_stream(V.psrow + tl.ps_begin + k, pol);
        }
      }
      // walk: a pseudo-row's sum is stored at its last nonzero (a predicated
      // store), a row end resets the running sum.  A pseudo-row begun in an
      // earlier lane and ended here (the head) gets the earlier lanes' part
      // below; one still open at the window's end goes to the scan
      const uint32_t d = cur.d;
      // lanes past the tile's end hold no nonzeros (d = 0: no row ends)
      const bool active = lane * 8 < tl.nz_len;
      const int r0 = (int)(d >> 17);
      int r = r0;
      float acc = 0.f;
      {
        float g[8], a[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) g[e] = vs[col16(cur.cc, e)];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          a[e] = cur.a0.v[e];
          a[4 + e] = cur.a1.v[e];
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          acc = fmaf(a[e], g[e], acc);
          if ((d >> e) & 1u) {
            st[r] = acc;
            acc = 0.f;
            ++r;
          }
        }
      }
      const int key = (active && !((d >> 7) & 1u)) ? r : -1;  // pseudo-row open at the window's end
      const int head_row = (active && ((d >> 16) & 1u) && (d & 0xffu)) ? r0 : -1;
      // the tile's values, columns and gathers are dead: the next tile's loads
      // go out now and overlap the scan, the head fix-up and the staged writes
      {
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(next_tile, 1);
        nxt = __shfl_sync(0xffffffffu, nxt, 0);
        t_next = nxt;
        if (nxt < bd.t_end) panel_load(cur, V, dc, bd.t_begin, nxt, lane, pol);
      }
      // segmented inclusive scan of the open sums (equal keys are adjacent lanes)
      float sv = acc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float up = __shfl_up_sync(0xffffffffu, sv, o);
        const int ku = __shfl_up_sync(0xffffffffu, key, o);
        if (lane >= o && ku == key && key >= 0) sv += up;
      }
      const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
      const float cprev = __shfl_up_sync(0xffffffffu, sv, 1);
      __syncwarp();
      if (head_row >= 0) {
        float head_val = st[head_row];  // this lane's part, stored at the row's end
        if (lane > 0 && kprev == head_row) head_val += cprev;
        st[head_row] = head_val;
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < kPanelPsCap / 32; ++j) {
        if (32 * j < nps) {
          const int k = lane + 32 * j;
          if (k < nps) part[rid[j]] = st[k];
        }
      }
      __syncwarp();
    }
    if (t_next < 0) {  // a long tile: the next tile's loads go out here
      int nxt = 0;
      if (lane == 0) nxt = atomicAdd(next_tile, 1);
      t_next = __shfl_sync(0xffffffffu, nxt, 0);
      if (t_next < bd.t_end) panel_load(cur, V, dc, bd.t_begin, t_next, lane, pol);
    }
    t = t_next;
  }
}

// Row pass: s_i = the sum of partial[p][i] over the panels in panel order,
// then the half-step's row epilogue.
// G = 0 (up to 32 panels, rows enough for 4 per thread on every SM): a
// thread takes 4 consecutive rows with 16-byte loads of each panel's 4 sums
// and of the epilogue's operands; rows past the last multiple of 4 one per
// thread.
// G >= 1: G consecutive lanes share a row: lane k adds its contiguous share
// of the panels in order (8 loads in flight per round), lane 0 adds the
// shares in lane order; warps stride over groups of 32 / G rows.
// The step's scalars (read by thread 0 into rs) are needed only to apply the
// epilogue: each thread first loads and adds its first rows' operands and
// sums, then meets the block barrier that publishes rs, so those loads
// overlap thread 0's read.  The epilogue is built with first = false (its
// loads do not skip the running average) and gets the scalars after the
// barrier.

// the step's scalars into the epilogue: a = tau or sigma, b = the averaging
// weight (or lam of the Halpern method)
struct RowScalars {
  float a, b;
  int first, done;
};
__device__ __forceinline__ void set_step(PrimalEpi<float>& e, const RowScalars& r) {
  e.tau = r.a;
  e.w = r.b;
  e.first = r.first != 0;
}
__device__ __forceinline__ void set_step(DualEpi<float>& e, const RowScalars& r) {
  e.sigma = r.a;
  e.w = r.b;
  e.first = r.first != 0;
}
__device__ __forceinline__ void set_step(HalpernPrimalEpi<float>& e, const RowScalars& r) {
  e.tau = r.a;
  e.lam = r.b;
}
__device__ __forceinline__ void set_step(HalpernDualEpi<float>& e, const RowScalars& r) {
  e.sigma = r.a;
  e.lam = r.b;
}

// the panels' sums of rows i..i+3, added in panel order
__device__ __forceinline__ float4 sum4(const PanelView& V, int i) {
  const int np = V.npanels;
  const size_t stride = (size_t)V.pstride;
  const float* pp = V.partial + i;
  float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int c = 0; c < np; c += 8) {
    float4 u[8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
      u[r] = c + r < np ? __ldcg(reinterpret_cast<const float4*>(pp + (size_t)(c + r) * stride))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if (c + r < np) {
        t.x += u[r].x;
        t.y += u[r].y;
        t.z += u[r].z;
        t.w += u[r].w;
      }
  }
  return t;
}

template <int G, class Epi>
__device__ __forceinline__ void panel_rows(const PanelView& V, Epi& epi, const RowScalars* rs) {
  const int rows = V.rows, np = V.npanels;
  const size_t stride = (size_t)V.pstride;
  if constexpr (G == 0) {
    const int nthr = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int n4 = rows >> 2;
    // the first quad of rows before the barrier
    typename Epi::In4 in0{};
    float4 t0 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid < n4) {
      in0 = epi.load4(tid << 2);
      t0 = sum4(V, tid << 2);
    }
    __syncthreads();
    if (rs->done) return;
    set_step(epi, *rs);
    if (tid < n4) epi.apply4(tid << 2, in0, t0);
    for (int q = tid + nthr; q < n4; q += nthr) {
      const int i = q << 2;
      const typename Epi::In4 in = epi.load4(i);
      epi.apply4(i, in, sum4(V, i));
    }
    for (int i = (n4 << 2) + tid; i < rows; i += nthr) {
      const typename Epi::In in = epi.load(i);
      float t = 0.f;
      for (int c = 0; c < np; ++c) t += __ldcg(V.partial + (size_t)c * stride + i);
      epi.apply(i, in, t);
    }
  } else {
    const int per = (np + G - 1) / G;  // panels of one lane
    const int lane = threadIdx.x & 31, k = lane % G, base_lane = lane - k;
    const int mine = max(0, min(per, np - k * per));
    const float* __restrict__ part = V.partial + (size_t)(k * per) * stride;
    constexpr int kRowsPerWarp = 32 / G;
    const int nw = gridDim.x * (blockDim.x >> 5);
    int r0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kRowsPerWarp;
    // one group of rows: the epilogue's operands and the row's sum (in lane 0 of the row)
    auto group = [&](int rr0, typename Epi::In& in, float& s) {
      const int i = rr0 + lane / G;
      const bool live = i < rows;
      if (live && k == 0) in = epi.load(i);
      float t = 0.f;
      const float* pp = part + i;
      for (int c = 0; c < mine; c += 8) {
        float q[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) q[r] = (live && c + r < mine) ? __ldcg(pp + (c + r) * stride) : 0.f;
#pragma unroll
        for (int r = 0; r < 8; ++r)
          if (c + r < mine) t += q[r];
      }
      s = t;
#pragma unroll
      for (int o = 1; o < G; ++o) {
        const float u = __shfl_sync(0xffffffffu, t, base_lane + o);
        if (k == 0) s += u;
      }
    };
    typename Epi::In in0{};
    float s0 = 0.f;
    if (r0 < rows) group(r0, in0, s0);  // warp-uniform
    __syncthreads();
    if (rs->done) return;
    set_step(epi, *rs);
    if (r0 < rows && r0 + lane / G < rows && k == 0) epi.apply(r0 + lane / G, in0, s0);
    for (r0 += nw * kRowsPerWarp; r0 < rows; r0 += nw * kRowsPerWarp) {
      typename Epi::In in{};
      float s = 0.f;
      group(r0, in, s);
      const int i = r0 + lane / G;
      if (i < rows && k == 0) epi.apply(i, in, s);
    }
  }
}

// The step's scalars, read from the device state by thread 0 (no barrier:
// panel_rows meets it after its first loads): a = tau or sigma, b = the
// averaging weight 1/(t+1) (or lam of the Halpern method), first = no
// average yet, done = the solve has finished.
__device__ __forceinline__ void row_scalars(const IterBuffers<float>& B, int i, bool dual,
                                            bool halpern, RowScalars* out) {
  if (threadIdx.x == 0) {
    const Scalars* sc = B.sc;
    const long long tt = sc->t + i;  // iterations since restart before this one
    out->done = sc->done;
    out->a = (float)(dual ? sc->sigma : sc->tau);
    out->b = halpern ? (float)((double)(tt + 1) / (double)(tt + 2)) : (float)(1.0 / (double)(tt + 1));
    out->first = tt == 0;
  }
}

template <int G>
// The row passes let the next kernel (the other half-step's panel SpMV) start
// its blocks as SMs free up: its prologue (tile descriptors, the L2 prefetch
// of its nonzeros, the first tile's loads) overlaps the end of the row pass
// (solve iteration 48.6 -> 46.8 us on the power-law LP).  The same early
// start of the row pass from the SpMV cost 1.4 us per iteration, and of the
// CSR tile kernels (no prologue) 7%, so those kernels do not trigger.
__global__ void __launch_bounds__(256, 6) k_panel_primal(IterBuffers<float> B, PanelView V, int i) {
  __shared__ RowScalars rs;
  pdl_trigger();
  pdl_enter();
  row_scalars(B, i, false, false, &rs);
  PrimalEpi<float> epi{B.x, B.c_t, B.x_avg, 0.f, 0.f, false};
  panel_rows<G>(V, epi, &rs);
}

template <int G>
__global__ void __launch_bounds__(256, 6) k_panel_dual(IterBuffers<float> B, PanelView V, int i) {
  __shared__ RowScalars rs;
  pdl_trigger();
  pdl_enter();
  row_scalars(B, i, true, false, &rs);
  DualEpi<float> epi{B.y, B.b_t, B.Ax, B.y_avg, B.Ax_avg, 0.f, 0.f, false};
  panel_rows<G>(V, epi, &rs);
}

template <int G>
__global__ void __launch_bounds__(256, 6) k_panel_hprimal(IterBuffers<float> B, PanelView V, int i) {
  __shared__ RowScalars rs;
  pdl_trigger();
  pdl_enter();
  row_scalars(B, i, false, true, &rs);
  HalpernPrimalEpi<float> epi{B.x, B.x_avg, B.c_t, B.x_last, 0.f, 0.f, (float)B.rho};
  panel_rows<G>(V, epi, &rs);
}

template <int G>
__global__ void __launch_bounds__(256, 6) k_panel_hdual(IterBuffers<float> B, PanelView V, int i) {
  __shared__ RowScalars rs;
  pdl_trigger();
  pdl_enter();
  row_scalars(B, i, true, true, &rs);
  HalpernDualEpi<float> epi{B.y,      B.b_t,     B.Ax, B.y_avg, B.Ax_avg,
                            B.y_last, B.Ax_last, 0.f,  0.f,     (float)B.rho};
  panel_rows<G>(V, epi, &rs);
}

// lanes per row: one up to 32 panels (each costs a lane a load and an add,
// fewer than sharing a row's overhead would), then enough that a lane holds
// at most 32 panels
int panel_lanes(int np) {
  int g = 1;
  while (g < 32 && g * 32 < np) g *= 2;
  return g;
}

// lanes per row of the row pass, 0 for 4 rows per thread: with up to 32 panels
// and at least 2^19 rows (enough threads to fill every SM at 4 rows each)
int row_lanes(int rows, int np) {
  const int g = panel_lanes(np);
  return g == 1 && rows >= (1 << 19) ? 0 : g;
}

#define PDHG_DISPATCH_G(g, ...)      \
  switch (g) {                       \
    case 0: {                        \
      constexpr int G_ = 0;          \
      __VA_ARGS__;                   \
    } break;                         \
    case 1: {                        \
      constexpr int G_ = 1;          \
      __VA_ARGS__;                   \
    } break;                         \
    case 2: {                        \
      constexpr int G_ = 2;          \
      __VA_ARGS__;                   \
    } break;                         \
    case 4: {                        \
      constexpr int G_ = 4;          \
      __VA_ARGS__;                   \
    } break;                         \
    case 8: {                        \
      constexpr int G_ = 8;          \
      __VA_ARGS__;                   \
    } break;                         \
    case 16: {                       \
      constexpr int G_ = 16;         \
      __VA_ARGS__;                   \
    } break;                         \
    default: {                       \
      constexpr int G_ = 32;         \
      __VA_ARGS__;                   \
    } break;                         \
  }

size_t panel_smem(int P, int pscap) {
  return sizeof(float) *
         ((size_t)kPanelWarps * pscap + 4 * (size_t)kPanelDescCache + 4 + (size_t)P);
}

// static shared memory of k_panel_spmv (its transaction barrier): the panel
// width leaves room for it below the opt-in limit
static size_t panel_static_smem() {
  static size_t bytes = [] {
    cudaFuncAttributes fa{};
    return cudaFuncGetAttributes(&fa, k_panel_spmv) == cudaSuccess ? fa.sharedSizeBytes : size_t(64);
  }();
  return bytes;
}

void launch_panel_half(const IterBuffers<float>& B, const PanelView& V, bool dual, int method,
                       int row_grid, int i, cudaStream_t s, cudaEvent_t between) {
  const float* v = dual ? (method == 1 ? B.x_avg : B.x) : B.y;
  launch_pdl(k_panel_spmv, V.nblocks, kPanelThreads, panel_smem(V.P, V.pscap), s, V, v,
             (const Scalars*)B.sc);
  if (between) cudaEventRecordWithFlags(between, s, cudaEventRecordExternal);
  const int g = row_lanes(V.rows, V.npanels);
  if (dual && method == 1) {
    PDHG_DISPATCH_G(g, launch_pdl(k_panel_hdual<G_>, row_grid, 256, 0, s, B, V, i));
  } else if (dual) {
    PDHG_DISPATCH_G(g, launch_pdl(k_panel_dual<G_>, row_grid, 256, 0, s, B, V, i));
  } else if (method == 1) {
    PDHG_DISPATCH_G(g, launch_pdl(k_panel_hprimal<G_>, row_grid, 256, 0, s, B, V, i));
  } else {
    PDHG_DISPATCH_G(g, launch_pdl(k_panel_primal<G_>, row_grid, 256, 0, s, B, V, i));
  }
}

void launch_panel_spmv_only(const IterBuffers<float>& B, const PanelView& V, bool dual, int method,
                            cudaStream_t s) {
  const float* v = dual ? (method == 1 ? B.x_avg : B.x) : B.y;
  launch_pdl(k_panel_spmv, V.nblocks, kPanelThreads, panel_smem(V.P, V.pscap), s, V, v,
             (const Scalars*)B.sc);
}

int panel_row_grid(int rows, int npanels, int nsm) {
  const int g = row_lanes(rows, npanels);
  const int64_t threads = g == 0 ? ((int64_t)rows + 3) / 4 : (int64_t)rows * g;
  return (int)std::max<int64_t>(1, std::min<int64_t>((threads + 255) / 256, (int64_t)nsm * 6));
}

cudaError_t configure_panel_kernels(size_t max_smem) {
  return set_max_dyn_smem((const void*)k_panel_spmv, max_smem);
}

// ---------------------------------------------------------------------------
// Layout build (device, once per context after scaling)
// ---------------------------------------------------------------------------
namespace {

// cnt[p*R + i] = nonzeros of row i in panel p, src[.] = the first of them
__global__ void k_pl_count(int R, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           int P, int32_t* cnt, int32_t* src) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < R; i += nw) {
    const int s = rp[i], e = rp[i + 1];
    for (int k = s + lane; k < e; k += 32) {
      const int p = col[k] / P;
      const int64_t f = (int64_t)p * R + i;
      atomicAdd(cnt + f, 1);
      if (k == s || col[k - 1] / P != p) src[f] = k;
    }
  }
}

__global__ void k_pl_flag(int64_t len, const int32_t* __restrict__ cnt, int32_t* flag) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < len;
       f += (int64_t)gridDim.x * blockDim.x)
    flag[f] = cnt[f] > 0;
}

__global__ void k_pl_compact(int64_t len, int R, const int32_t* __restrict__ cnt,
                             const int32_t* __restrict__ src, const int32_t* __restrict__ psidx,
                             int32_t* psrow, int32_t* pslen, int32_t* pssrc) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < len;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int c = cnt[f];
    if (c > 0) {
      const int k = psidx[f];
      psrow[k] = (int32_t)(f % R);
      pslen[k] = c;
      pssrc[k] = src[f];
    }
  }
}

// out[p] = psidx[p * R] for p = 0..np (the first pseudo-row of each panel)
__global__ void k_pl_panel_first(int np, int R, const int32_t* __restrict__ psidx, int32_t* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p <= np) out[p] = psidx[(int64_t)p * R];
}

// greedy packing of a segment of one panel's pseudo-rows into warp tiles;
// emit = false only counts them
// tile packing: segments of at most kPackSeg pseudo-rows, kPackWarps per block
constexpr int kPackSeg = 2048, kPackWarps = 4;

template <bool kEmit>
__global__ void __launch_bounds__(kPackWarps * 32)
    k_pl_pack(int nseg, const int2* __restrict__ segs, const int32_t* __restrict__ seg_panel,
              const int32_t* __restrict__ pslen, const int32_t* __restrict__ toff, int pscap,
              int32_t* tcount, PanelTile* tiles, int32_t* tlen, int32_t* tpanel) {
  // a warp per segment: its pseudo-row lengths go to shared memory with
  // coalesced loads, then lane 0 packs them greedily in order
  __shared__ int32_t sl[kPackWarps][kPackSeg];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * kPackWarps + w;
  if (s >= nseg) return;  // warp-uniform
  const int b = segs[s].x, e = segs[s].y;
  int32_t* len = sl[w] - b;  // len[k] = pslen[k] for b <= k < e
  for (int k = b + lane; k < e; k += 32) len[k] = pslen[k];
  __syncwarp();
  if (lane != 0) return;
  int nt = 0, k = b;
  while (k < e) {
    const int L = len[k];
    PanelTile tl{0, 0, k, 0};
    if (L > kPanelCap) {
      tl.nz_len = (L + 7) & ~7;
      tl.nps = -1;
      ++k;
    } else {
      int used = 0;
      while (k < e && len[k] <= kPanelCap && used + len[k] <= kPanelCap &&
             k - tl.ps_begin < pscap)
        used += len[k++];
      tl.nz_len = (used + 7) & ~7;
      tl.nps = k - tl.ps_begin;
    }
    if (kEmit) {
      const int t = toff[s] + nt;
      tiles[t] = tl;
      tlen[t] = tl.nz_len;
      tpanel[t] = seg_panel[s];
    }
    ++nt;
  }
  if (!kEmit) tcount[s] = nt;
}

__global__ void k_pl_tile_begin(int nt, const int32_t* __restrict__ nzoff, PanelTile* tiles) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nt) tiles[t].nz_begin = nzoff[t];
}

// values, panel columns and window words of every tile (a warp per tile)
__global__ void k_pl_fill(int nt, const PanelTile* __restrict__ tiles,
                          const int32_t* __restrict__ tpanel, const int32_t* __restrict__ pslen,
                          const int32_t* __restrict__ pssrc, const int32_t* __restrict__ col,
                          const float* __restrict__ val, int P, float* val_p, uint16_t* col_p,
                          uint32_t* wd_p) {
  __shared__ int start_s[8][kPanelCap + 1];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  int* start = start_s[wib];
  for (int t = warp; t < nt; t += nw) {
    const PanelTile tl = tiles[t];
    const int c0 = tpanel[t] * P;
    const int nz = tl.nz_begin;
    if (tl.nps < 0) {
      const int L = pslen[tl.ps_begin], s0 = pssrc[tl.ps_begin];
      for (int q = lane; q < tl.nz_len; q += 32) {
        val_p[nz + q] = q < L ? val[s0 + q] : 0.f;
        col_p[nz + q] = q < L ? (uint16_t)(col[s0 + q] - c0) : (uint16_t)0;
      }
      for (int w = lane; w < tl.nz_len / 8; w += 32) wd_p[nz / 8 + w] = 0u;
      continue;
    }
    // starts of the pseudo-rows within the tile: lane l sums pseudo-rows 8l..8l+7
    int loc[8], tot = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = 8 * lane + j;
      loc[j] = tot;
      tot += k < tl.nps ? pslen[tl.ps_begin + k] : 0;
    }
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int up = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += up;
    }
    const int excl = incl - tot;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = 8 * lane + j;
      if (k < tl.nps) start[k] = excl + loc[j];
    }
    if (lane == 0) start[tl.nps] = tl.nz_len;  // the last pseudo-row absorbs the padding
    __syncwarp();
    for (int q = lane; q < tl.nz_len; q += 32) {
      int lo = 0, hi = tl.nps - 1;  // last pseudo-row with start <= q
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= q) lo = mid;
        else hi = mid - 1;
      }
      const int off = q - start[lo];
      const bool real = off < pslen[tl.ps_begin + lo];
      const int sidx = pssrc[tl.ps_begin + lo] + off;
      val_p[nz + q] = real ? val[sidx] : 0.f;
      col_p[nz + q] = real ? (uint16_t)(col[sidx] - c0) : (uint16_t)0;
    }
    for (int w = lane; w < tl.nz_len / 8; w += 32) {
      const int q0 = 8 * w;
      int lo = 0, hi = tl.nps - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= q0) lo = mid;
        else hi = mid - 1;
      }
      const uint32_t head = start[lo] < q0 ? 1u : 0u;
      uint32_t mask = 0u;
      int j = lo;
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (q0 + e == start[j + 1] - 1) {
          mask |= 1u << e;
          ++j;
        }
      wd_p[nz / 8 + w] = ((uint32_t)lo << 17) | (head << 16) | mask;
    }
    __syncwarp();
  }
}

int grid_for(int64_t work, int per = 256, int cap = 16384) {
  int64_t g = (work + per - 1) / per;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

template <typename T>
struct Tmp {  // device scratch freed with the object
  T* p = nullptr;
  ~Tmp() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t n) { return cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)); }
};

}  // namespace

bool panel_shape(const pdhg_ctx* ctx, bool on_a, int* P_out, int* np_out, int pscap) {
  if (!ctx->mixed || ctx->batch || ctx->nnz < 1) return false;
  const int64_t R = on_a ? ctx->m : ctx->n, C = on_a ? ctx->n : ctx->m;
  if (R < 1 || C < 1 || ctx->nnz > (int64_t(1) << 30)) return false;
  const int64_t dyn = (int64_t)ctx->smem_optin - (int64_t)panel_static_smem();
  int64_t pmax = (dyn / (int64_t)sizeof(float) - (int64_t)kPanelWarps * pscap -
                  4 * kPanelDescCache - 4) &
                 ~int64_t(7);
  pmax = std::min<int64_t>(pmax, 65536);
  if (pmax < 1024) return false;
  if (ctx->opt.panel_width > 0) pmax = std::min<int64_t>(pmax, std::max(8, ctx->opt.panel_width & ~7));
  const int64_t np = (C + pmax - 1) / pmax;
  const int64_t P = (((C + np - 1) / np) + 7) & ~int64_t(7);
  // the partial sums are dense over (panel, row): at most about twice the nonzeros
  if (np * R > 2 * ctx->nnz + R || np * R >= (int64_t(1) << 31) - 1024) return false;
  *P_out = (int)P;
  *np_out = (int)np;
  return true;
}

#define PL_CK(x)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (x);                                                         \
    if (e_ != cudaSuccess) {                                                      \
      set_error("panel layout: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? PDHG_OOM : PDHG_CUDA_ERROR;        \
    }                                                                             \
  } while (0)

pdhg_status build_panel_layout(pdhg_ctx* ctx, bool on_a, DevPanel* out) {
  *out = DevPanel{};
  int P = 0, np = 0;
  if (!panel_shape(ctx, on_a, &P, &np, 256)) {
    set_error("column panels do not apply to this matrix");
    return PDHG_INVALID_ARG;
  }
  cudaStream_t s = ctx->stream;
  const int R = on_a ? ctx->m : ctx->n, C = on_a ? ctx->n : ctx->m;
  const int32_t* rp = on_a ? ctx->a_rp : ctx->t_rp;
  const int32_t* col = on_a ? ctx->a_col : ctx->t_col;
  const float* val = on_a ? ctx->a_val32 : ctx->t_val32;
  int64_t len = (int64_t)np * R;  // the 256 cap gives the narrowest panels: the most of them
  const int pstride = (R + 3) & ~3;

  // pseudo-rows: counts per (panel, row), their prefix, the first of each panel
  Tmp<int32_t> cnt, src, flag, psidx, scan_tmp, pfirst;
  PL_CK(cnt.alloc(len));
  PL_CK(src.alloc(len));
  PL_CK(flag.alloc(len));
  PL_CK(psidx.alloc(len + 1));
  PL_CK(scan_tmp.alloc(len / 1024 + 2 + 1024));
  PL_CK(pfirst.alloc(np + 1));
  std::vector<int32_t> h_pfirst;
  auto count = [&](int P_, int np_) -> pdhg_status {
    const int64_t len_ = (int64_t)np_ * R;
    PL_CK(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * len_, s));
    k_pl_count<<<grid_for((int64_t)R * 32), 256, 0, s>>>(R, rp, col, P_, cnt.p, src.p);
    k_pl_flag<<<grid_for(len_), 256, 0, s>>>(len_, cnt.p, flag.p);
    launch_scan(flag.p, psidx.p, (int)len_, scan_tmp.p, s);
    k_pl_panel_first<<<(np_ + 256) / 256, 256, 0, s>>>(np_, R, psidx.p, pfirst.p);
    h_pfirst.assign(np_ + 1, 0);
    PL_CK(cudaMemcpyAsync(h_pfirst.data(), pfirst.p, sizeof(int32_t) * (np_ + 1),
                          cudaMemcpyDeviceToHost, s));
    PL_CK(cudaStreamSynchronize(s));
    ctx->launches += 6;
    return PDHG_OK;
  };
  CKS(count(P, np));
  // A tile holds at most 256 nonzeros: when it holds fewer than 96 pseudo-rows
  // on average, a cap of 128 pseudo-rows rarely binds, and the halved staging
  // of the sums buys wider panels (fewer panels, pseudo-rows and partial sums).
  int pscap = 256, P128 = 0, np128 = 0;
  if ((double)kPanelCap * (double)h_pfirst[np] < 96.0 * (double)ctx->nnz &&
      panel_shape(ctx, on_a, &P128, &np128, 128) && P128 != P) {
    pscap = 128;
    P = P128;
    np = np128;
    len = (int64_t)np * R;
    CKS(count(P, np));
  }
  const int nps = h_pfirst[np];
  CKS(dalloc(ctx, &out->psrow, (size_t)nps + 16));  // spare: prefetches round up to 16 bytes
  Tmp<int32_t> pslen, pssrc;
  PL_CK(pslen.alloc(nps));
  PL_CK(pssrc.alloc(nps));
  k_pl_compact<<<grid_for(len), 256, 0, s>>>(len, R, cnt.p, src.p, psidx.p, out->psrow, pslen.p,
                                             pssrc.p);

  // segments of at most kPackSeg pseudo-rows within a panel, packed in parallel
  constexpr int kSeg = kPackSeg;
  std::vector<int2> h_segs;
  std::vector<int32_t> h_seg_panel;
  for (int p = 0; p < np; ++p)
    for (int b = h_pfirst[p]; b < h_pfirst[p + 1]; b += kSeg) {
      h_segs.push_back(make_int2(b, std::min(b + kSeg, h_pfirst[p + 1])));
      h_seg_panel.push_back(p);
    }
  const int nseg = (int)h_segs.size();
  Tmp<int2> segs;
  Tmp<int32_t> seg_panel, tcount, toff;
  PL_CK(segs.alloc(nseg));
  PL_CK(seg_panel.alloc(nseg));
  PL_CK(tcount.alloc(nseg));
  PL_CK(toff.alloc(nseg + 1));
  if (nseg > 0) {
    PL_CK(cudaMemcpyAsync(segs.p, h_segs.data(), sizeof(int2) * nseg, cudaMemcpyHostToDevice, s));
    PL_CK(cudaMemcpyAsync(seg_panel.p, h_seg_panel.data(), sizeof(int32_t) * nseg,
                          cudaMemcpyHostToDevice, s));
    k_pl_pack<false><<<(nseg + kPackWarps - 1) / kPackWarps, kPackWarps * 32, 0, s>>>(nseg, segs.p, seg_panel.p, pslen.p,
                                                         nullptr, pscap, tcount.p, nullptr, nullptr,
                                                         nullptr);
  }
  launch_scan(tcount.p, toff.p, nseg, scan_tmp.p, s);
  std::vector<int32_t> h_toff(nseg + 1);
  PL_CK(cudaMemcpyAsync(h_toff.data(), toff.p, sizeof(int32_t) * (nseg + 1),
                        cudaMemcpyDeviceToHost, s));
  PL_CK(cudaStreamSynchronize(s));
  const int nt = h_toff[nseg];
  CKS(dalloc(ctx, &out->tiles, (size_t)nt));
  Tmp<int32_t> tlen, tpanel, nzoff;
  PL_CK(tlen.alloc(nt));
  PL_CK(tpanel.alloc(nt));
  PL_CK(nzoff.alloc(nt + 1));
  if (nseg > 0)
    k_pl_pack<true><<<(nseg + kPackWarps - 1) / kPackWarps, kPackWarps * 32, 0, s>>>(nseg, segs.p, seg_panel.p, pslen.p, toff.p,
                                                        pscap, nullptr, out->tiles, tlen.p, tpanel.p);
  launch_scan(tlen.p, nzoff.p, nt, scan_tmp.p, s);
  if (nt > 0) k_pl_tile_begin<<<(nt + 255) / 256, 256, 0, s>>>(nt, nzoff.p, out->tiles);
  std::vector<int32_t> h_nzoff(nt + 1);
  PL_CK(cudaMemcpyAsync(h_nzoff.data(), nzoff.p, sizeof(int32_t) * (nt + 1),
                        cudaMemcpyDeviceToHost, s));
  PL_CK(cudaStreamSynchronize(s));
  const int64_t nzp = h_nzoff[nt];
  ctx->launches += 10;

  CKS(dalloc(ctx, &out->val, (size_t)nzp + 16));
  CKS(dalloc(ctx, &out->col, (size_t)nzp + 32));
  CKS(dalloc(ctx, &out->wd, (size_t)nzp / 8 + 16));
  if (nt > 0)
    k_pl_fill<<<grid_for((int64_t)nt * 32), 256, 0, s>>>(nt, out->tiles, tpanel.p, pslen.p, pssrc.p,
                                                        col, val, P, out->val, out->col, out->wd);
  ctx->launches += 1;

  // blocks: one per SM (or per panel when there are more panels), apportioned
  // to the panels by their nonzeros, each a contiguous range of its panel's tiles
  std::vector<int> pt_begin(np, 0), pt_end(np, 0);
  {
    int sidx = 0;
    for (int p = 0; p < np; ++p) {
      pt_begin[p] = h_toff[sidx];
      while (sidx < nseg && h_seg_panel[sidx] == p) ++sidx;
      pt_end[p] = h_toff[sidx];
    }
  }
  std::vector<int64_t> pnz(np);
  int nonempty = 0;
  int64_t tot = 0;
  for (int p = 0; p < np; ++p) {
    pnz[p] = h_nzoff[pt_end[p]] - h_nzoff[pt_begin[p]];
    tot += pnz[p];
    nonempty += pnz[p] > 0;
  }
  const int nb_total = std::max(ctx->nsm, nonempty);
  std::vector<int> nbp(np, 0);
  {
    int left = nb_total;
    std::vector<std::pair<double, int>> rem;
    for (int p = 0; p < np; ++p) {
      if (pnz[p] == 0) continue;
      const double q = (double)nb_total * (double)pnz[p] / (double)std::max<int64_t>(tot, 1);
      nbp[p] = std::max(1, (int)q);
      left -= nbp[p];
      rem.push_back({q - (int)q, p});
    }
    std::sort(rem.begin(), rem.end(),
              [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
                return a.first > b.first || (a.first == b.first && a.second < b.second);
              });
    for (size_t r = 0; left > 0 && r < rem.size(); ++r, --left) nbp[rem[r].second]++;
  }
  std::vector<PanelBlock> h_blocks;
  for (int p = 0; p < np; ++p) {
    if (pnz[p] == 0) continue;
    int tb = pt_begin[p];
    const int64_t z0 = h_nzoff[pt_begin[p]];
    for (int b = 1; b <= nbp[p]; ++b) {
      int te = pt_end[p];
      if (b < nbp[p]) {
        const int64_t target = z0 + pnz[p] * b / nbp[p];
        te = (int)(std::lower_bound(h_nzoff.begin() + tb, h_nzoff.begin() + pt_end[p], target) -
                   h_nzoff.begin());
      }
      if (te > tb) {
        h_blocks.push_back(PanelBlock{p, tb, te, 0});
        tb = te;
      }
    }
  }
  const int nb = (int)h_blocks.size();
  CKS(dalloc(ctx, &out->blocks, (size_t)nb));
  if (nb > 0)
    PL_CK(cudaMemcpyAsync(out->blocks, h_blocks.data(), sizeof(PanelBlock) * nb,
                          cudaMemcpyHostToDevice, s));
  CKS(dalloc(ctx, &out->partial, (size_t)np * pstride));
  PL_CK(cudaMemsetAsync(out->partial, 0, sizeof(float) * (size_t)np * pstride, s));
  PL_CK(cudaStreamSynchronize(s));  // the host vectors above go out of scope
  PL_CK(cudaGetLastError());

  PanelView& V = out->view;
  V.tiles = out->tiles;
  V.blocks = out->blocks;
  V.val = out->val;
  V.col = out->col;
  V.wd = out->wd;
  V.psrow = out->psrow;
  V.partial = out->partial;
  V.P = P;
  V.npanels = np;
  V.rows = R;
  V.cols = C;
  V.nblocks = nb;
  V.ntiles = nt;
  V.pscap = pscap;
  V.pstride = pstride;
  if (!ctx->panel_err) {
    CKS(dalloc(ctx, &ctx->panel_err, 1));
    PL_CK(cudaMemsetAsync(ctx->panel_err, 0, sizeof(int32_t), s));
    PL_CK(cudaStreamSynchronize(s));
  }
  V.err = ctx->panel_err;
  V.tx_extra = ctx->opt.wait_test ? 16u : 0u;
  V.wait_ns = (unsigned long long)ctx->opt.wait_limit_ms * 1000000ull;
  out->pseudo_rows = nps;
  out->nnz_padded = nzp;
  out->on = nb > 0;
  return PDHG_OK;
}

}  // namespace pdhg
