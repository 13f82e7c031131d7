// Shared device-side definitions for the restarted-PDHG kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pdhg {

constexpr int kWarp = 32;

// ---------------------------------------------------------------------------
// CSR tile schedule.  A tile is a run of whole rows whose nonzeros fit in
// `tile_nnz`, one chunk of a row longer than that ("split row"), or a run of
// rows without nonzeros (nz_begin == nz_end).  A split row's chunks form a
// group: each chunk writes its partial sum to a slot, and the chunk that
// arrives last (atomic ticket) adds the slots in chunk order and runs the row
// epilogue, so the sum order is fixed.
// ---------------------------------------------------------------------------
struct Tile {
  int32_t row_begin, row_end;  // rows [row_begin, row_end)
  int32_t nz_begin, nz_end;    // nonzeros [nz_begin, nz_end)
  int32_t split;               // -1: whole rows; else split-group index
  int32_t part;                // chunk index within the split group
  int32_t lp;                  // LP of the tile's rows (batched solves; 0 otherwise)
  int32_t word0;               // segmented schedules: first window word of the tile
};

struct SplitGroup {
  int32_t row;
  int32_t nparts;
  int32_t slot0;  // first slot of this group in the slot array
  int32_t pad;
};

struct SchedView {
  const Tile* tiles;
  const SplitGroup* groups;
  int32_t* counters;  // [ngroups], zero between launches
  void* slots;        // [total parts * NV] partial sums
  const void* wd;      // window words of the whole-row tiles (segmented schedules)
  int32_t ntiles;
  int32_t tile_nnz;  // nonzero capacity of a tile (block * e - 4)
  int32_t max_rows;  // rows per tile at most
  int32_t ngroups;   // split groups (records appended after block partials)
  int32_t e;         // nonzeros per thread (4, 8 or 16)
  int32_t pad;
};

// ---------------------------------------------------------------------------
// Column-panel layout of one matrix (float32 iterations).  The columns are cut
// into panels of P; the nonzeros of row i inside panel p form pseudo-row
// (p, i).  Pseudo-rows are ordered by (panel, row) and packed whole into warp
// tiles of at most kPanelCap nonzeros and `pscap` (128 or 256) pseudo-rows,
// padded with zeros to a multiple of 8;
// a pseudo-row longer than kPanelCap is a tile of its own (nps < 0).  Each
// block stages one panel of the gathered vector in shared memory and runs a
// contiguous range of that panel's tiles; each pseudo-row's sum goes to
// partial[p * rows + i] (entries of empty pseudo-rows stay zero).
// ---------------------------------------------------------------------------
constexpr int kPanelWarps = 32;                 // warps of a panel block
constexpr int kPanelCap = 256;                  // nonzeros of a warp tile
constexpr int kPanelPsCap = 256;                // pseudo-rows of a warp tile, at most
constexpr int kPanelDescCache = 256;            // tile descriptors a block keeps in shared memory

struct PanelTile {
  int32_t nz_begin;  // first nonzero (a multiple of 8)
  int32_t nz_len;    // nonzeros incl. padding (a multiple of 8)
  int32_t ps_begin;  // first pseudo-row
  int32_t nps;       // pseudo-rows; -1: one pseudo-row longer than kPanelCap
};

struct PanelBlock {
  int32_t panel, t_begin, t_end, pad;
};

struct PanelView {
  const PanelTile* tiles;
  const PanelBlock* blocks;
  const float* val;     // [nonzeros incl. padding]
  const uint16_t* col;  // column within the panel
  const uint32_t* wd;   // window words, one per 8 nonzeros
  const int32_t* psrow; // row of each pseudo-row
  float* partial;       // [npanels][pstride]: panel p's sums at p * pstride + row
  int32_t P, npanels, rows, cols, nblocks, ntiles;
  int32_t pscap;        // pseudo-rows of a tile at most (128 or 256): the staged sums per warp
  int32_t pstride;      // rows rounded up to a multiple of 4 (16-byte aligned panels)
  int32_t* err;         // set to 1 when the panel load's bounded wait ran out
  uint32_t tx_extra;    // bytes the load expects beyond its copies (16 to test the bound, else 0)
  unsigned long long wait_ns;  // bound of the panel load's wait
};

// ---------------------------------------------------------------------------
// Device-resident solver scalars (float64 state of the restart rule).
// ---------------------------------------------------------------------------
enum { Q_S1 = 0,  // ||b~ - A~x||^2            (scaled primal residual)
       Q_S2,      // ||min(0, c~ - A~^T y)||^2  (scaled dual residual)
       Q_S3,      // c~^T x~ (= c^T x)
       Q_S4,      // b~^T y~ (= b^T y)
       Q_U1,      // ||b - Ax||^2  (original model)
       Q_U2,      // ||min(0, c - A^T y)||^2 (original model)
       Q_D1,      // ||x~ - x~_last||^2
       Q_D2,      // ||y~ - y~_last||^2
       Q_N };

struct Scalars {
  double omega, tau, sigma, eta;
  double kkt_last, kkt_prev;
  double norm_b, norm_c;        // original-model norms
  double eps;
  double beta_suff, beta_nec, beta_art, theta;
  double q[2][Q_N];             // last evaluation, [0] current, [1] average
  long long k, t, restarts, max_iter;
  int32_t eval_freq;
  int32_t done;                 // solve finished (kernels become no-ops)
  int32_t status;               // pdhg_status of the solve
  int32_t chosen_avg;           // returned iterate is the running average
  int32_t restart_pending;      // restart_apply must act
  int32_t restart_to_avg;       // ... with the average as the new iterate
  int32_t log_count, log_cap;
  int32_t ticket;               // last-block-done counter for the eval kernel
  int32_t pad;
  // float32-mixed: a Section 2 test that passes on the float32 caches is a
  // screen; the candidate is then re-evaluated in float64 (products
  // recomputed from the float64 scaled matrices) and only that decides
  double screen;                // the screen passes at eps * screen (>= 1)
  long long checks, rejects;    // float64 checks run / rejected in this solve
  int32_t fp64_check;           // 1: confirm a passing screen in float64
  int32_t verify;               // 1: a float64 check is pending
  int32_t verify_avg;           // ... of the average (1) or the current iterate (0)
  int32_t omega_rule;           // 0: smoothing with theta; 1: PID control of log omega
  double pid_kp, pid_ki, pid_kd;
  double pid_integral, pid_prev;  // sum of the PID errors so far, the last error
  // adaptive step (step_rule 1, PDLP's rule): eta is the next attempt's step,
  // eta_sum the accepted steps since the last restart, avg_w / avg_first the
  // next attempt's averaging weight eta / (eta_sum + eta) and "no average yet",
  // accept the last attempt's decision
  int32_t step_rule;
  int32_t accept;
  int32_t avg_first;
  int32_t pad2;
  double avg_w;
  double eta_sum;
  long long step_rejects;
};

struct PowerState {
  double lam, lam_prev, inv_norm;
  int32_t k, max_iter, stopped, ticket;
  double rel_tol;
};

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// The block's sums of NQ float64 quantities (each thread holds its share in
// v), written to out[0..NQ) by threads 0..NQ-1.  Within a warp the sums are
// reduce-scattered: at each of the five shuffle steps a lane keeps half of
// the quantities it still holds and adds its partner's half of the same ones
// (then, one quantity left, the partner's value), so a lane adds NQ + 1
// values rather than the 5 NQ of block_sum below (GB300's float64 pipe makes
// that difference count for NQ = 16).  Lane l ends with the warp's sum of
// quantity l >> (5 - log2 NQ); the warps' sums are added in warp order.  The
// order is fixed, so the sums do not depend on scheduling.  Called by every
// thread of the block; `red` holds NQ * (BLOCK / 32) doubles of shared
// memory; ends with a block barrier (a fence by one thread after it covers
// the block's writes to out).
template <int NQ>
constexpr int log2_of() {
  return NQ <= 1 ? 0 : 1 + log2_of<NQ / 2>();
}
template <int BLOCK, int NQ>
__device__ __forceinline__ void block_sum_scatter(double (&v)[NQ], double* red, double* out) {
  static_assert(NQ >= 1 && NQ <= 32 && (NQ & (NQ - 1)) == 0 && BLOCK % 32 == 0, "NQ");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int o = 16 >> st;
    if ((NQ >> st) >= 2) {
      const int half = (NQ >> st) / 2;
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int k = 0; k < NQ / 2; ++k) {
        if (k < half) {
          const double send = up ? v[k] : v[k + half];
          const double keep = up ? v[k + half] : v[k];
          v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    }
  }
  constexpr int kShift = 5 - log2_of<NQ>();
  if ((lane & ((1 << kShift) - 1)) == 0) red[w * NQ + (lane >> kShift)] = v[0];
  __syncthreads();
  if (threadIdx.x < NQ) {
    double t = 0.0;
    for (int q = 0; q < BLOCK / 32; ++q) t += red[q * NQ + threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// Reduce `nq` doubles per thread over the block; result valid in thread 0's
// `out`.  `red` holds nq * (BLOCK / 32) doubles of shared memory.
template <int BLOCK, int NQ>
__device__ __forceinline__ void block_sum(const double (&v)[NQ], double (&out)[NQ], double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double s = warp_sum(v[q]);
    if (lane == 0) red[q * (BLOCK / 32) + w] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = 0.0;
      for (int i = 0; i < BLOCK / 32; ++i) s += red[q * (BLOCK / 32) + i];
      out[q] = s;
    }
  }
  __syncthreads();
}

// Sum of NQ-vectors stored one after another: parts a[0..na) then b[0..nb)
// (entry p holds NQ doubles), computed by every thread of one block in a
// fixed order: thread t sums entries t / NQ, t / NQ + BLOCK / NQ, ... of
// quantity t % NQ, then the threads of a quantity are combined by a fixed
// shuffle tree and the warps in order.  NQ a power of two <= 32 dividing
// BLOCK.  The result is in out[0..NQ) (shared) after the final barrier.
template <int BLOCK, int NQ>
__device__ __forceinline__ void parts_sum(const double* a, int na, const double* b, int nb,
                                          double* out, double* red) {
  static_assert(NQ >= 1 && NQ <= 32 && (NQ & (NQ - 1)) == 0 && BLOCK % 32 == 0, "NQ");
  constexpr int L = BLOCK / NQ;
  const int t = threadIdx.x, q = t % NQ, lane = t & 31, w = t >> 5;
  double s = 0.0;
  for (int p = t / NQ; p < na + nb; p += L)
    s += p < na ? __ldcg(a + (size_t)p * NQ + q) : __ldcg(b + (size_t)(p - na) * NQ + q);
#pragma unroll
  for (int o = 16; o >= NQ; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane < NQ) red[w * NQ + lane] = s;
  __syncthreads();
  if (t < NQ) {
    double v = 0.0;
    for (int i = 0; i < BLOCK / 32; ++i) v += red[i * NQ + t];
    out[t] = v;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Loads of the matrix stream (column indices, values, window words): read
// once per SpMV, so they carry an L2 evict-first policy and skip L1, leaving
// both caches to the gathered vector and the per-row operands.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t stream_policy() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ int4 ld_stream_int4(const int32_t* p, uint64_t pol) {
  int4 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p, uint64_t pol) {
  uint32_t r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ uint64_t ld_stream(const uint64_t* p, uint64_t pol) {
  uint64_t r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ int32_t ld_stream(const int32_t* p, uint64_t pol) {
  int32_t r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ float ld_stream(const float* p, uint64_t pol) {
  float r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ double ld_stream(const double* p, uint64_t pol) {
  double r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(pol));
  return r;
}

// Asynchronous L2 prefetch of [p, p + bytes) by the bulk-copy engine (one
// thread issues it; no registers wait on it).  The range is widened to 16-byte
// boundaries, so the array must have 16 bytes to spare past its end.
__device__ __forceinline__ void prefetch_l2(const void* p, int64_t bytes) {
  if (bytes <= 0) return;
  const uintptr_t lo = reinterpret_cast<uintptr_t>(p) & ~uintptr_t(15);
  const uintptr_t hi = (reinterpret_cast<uintptr_t>(p) + (uintptr_t)bytes + 15) & ~uintptr_t(15);
  for (uintptr_t a = lo; a < hi; a += 65536) {
    const uint32_t sz = (uint32_t)((hi - a) < 65536 ? (hi - a) : 65536);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(sz) : "memory");
  }
}

// Programmatic dependent launch: a half-step kernel launched with the
// programmatic-serialization attribute may become resident while the kernel
// before it drains; it lets its own successor do the same, then waits for
// its predecessor's completion (and memory) before reading anything.
// Launched without the attribute both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Lets the next kernel of the stream (launched with programmatic stream
// serialization) start its blocks as SMs free up, ahead of this grid's end.
// Its griddepcontrol.wait still waits for this whole grid to complete and
// flush, so only its prologue over constant data overlaps this kernel.  Every
// block of this grid calls it, so the next grid starts only after this one's
// last block is running (no block of this grid waits for an SM).
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Wall-clock time of the GPU in ns (bounds of device-side waits).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A shared-memory transaction barrier (mbarrier) for bulk copies into shared
// memory: one arrival (the thread that issues the copies) plus the bytes the
// copies deliver.  mb is the barrier's shared-memory address.
__device__ __forceinline__ void mbar_init(uint32_t mb) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint32_t mb, uint32_t bytes) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(mb),
               "r"(bytes)
               : "memory");
}
// global [src, src + bytes) -> shared dst (both 16-byte aligned, bytes a
// multiple of 16), completing on the barrier mb
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                              uint32_t mb) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mb)
      : "memory");
}
// waits for phase `parity` of the barrier to complete, at most limit_ns
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity, unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(mb), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }

// four consecutive values of the matrix stream (16- or 32-byte aligned)
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  float v[4];
  __device__ __forceinline__ void load_stream(const float* p, uint64_t pol) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
        : "l"(p), "l"(pol));
  }
};
template <> struct Vec4<double> {
  double v[4];
  __device__ __forceinline__ void load_stream(const double* p, uint64_t pol) {
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
        : "=d"(v[0]), "=d"(v[1])
        : "l"(p), "l"(pol));
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
        : "=d"(v[2]), "=d"(v[3])
        : "l"(p + 2), "l"(pol));
  }
};

}  // namespace pdhg
