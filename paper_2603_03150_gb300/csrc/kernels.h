// Host-side launchers for the PDHG kernels (implemented in *_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace pdhg {

constexpr int kBlock = 256;       // threads per block of every tile kernel
constexpr int kFixedE = 8;        // nonzeros per thread of the float64 report,
                                  // Algorithm 1 and power-iteration schedules
constexpr int kEvalQ = 2 * Q_N;   // reduced quantities per evaluation

// Device pointers of one LP's iteration state in precision T.
template <typename T>
struct IterBuffers {
  const int32_t *a_rp, *a_col;  // A~ (rows = m)
  const T* a_val;
  const int32_t *t_rp, *t_col;  // A~^T (rows = n)
  const T* t_val;
  SchedView a_sched, t_sched;
  // averaged method: x_avg, y_avg, Ax_avg are the running averages;
  // Halpern method: they hold T(z) = (x^, y^) and A~x^, and x_last, y_last,
  // Ax_last the anchor (last restart point) and its product
  T *x, *y, *x_avg, *y_avg, *x_last, *y_last, *Ax, *Ax_avg, *Ax_last;
  double rho;  // Halpern reflection
  const T *c_t, *b_t;                       // scaled c, b in precision T
  const double *c_t64, *b_t64, *D_r, *D_c;  // float64 copies and scalings
  const double *Dr_inv, *Dc_inv;            // their reciprocals
  Scalars* sc;
  // adaptive step (step_rule 1): the accepted state before an attempt (x in
  // adapt_xx), the attempt's iterate and the accepted one interleaved,
  // (x+_j, x_j) at 2j, 2j + 1 [2n], and the sums of the attempt: ||dx||^2
  // per block of the primal kernel [adapt_np] and per split row of A~^T,
  // then (||dy||^2, dy^T A~dx) per block of the dual kernel and per split
  // row of A~
  T *x_avg_prev, *y_prev, *y_avg_prev, *Ax_prev, *Ax_avg_prev;
  T* adapt_xx;
  double *adapt_pp, *adapt_sp, *adapt_pd, *adapt_sd;
  int adapt_np;
  double* partials;    // [grid][kEvalQ]
  double* split_q;     // [split groups of A^T][kEvalQ]
  long long* log_k;
  int32_t* log_flags;
  double* log_kkt;
  int32_t m, n;
};

// Nonzeros a context accepts: tiles index nonzeros with int32 and a window may
// reach 32 past the last one.
constexpr int64_t kMaxNnz = (int64_t(1) << 31) - (int64_t(1) << 16);

struct Launch {
  int grid;
  size_t smem;
};

// one PDHG iteration, iteration index i within the current chunk
template <typename T>
void launch_primal(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s);
template <typename T>
void launch_dual(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s);
// evaluation after `chunk` iterations + on-device restart/termination rule
template <typename T>
void launch_eval(const IterBuffers<T>& B, const Launch& L, int chunk, cudaStream_t s);
template <typename T>
void launch_restart(const IterBuffers<T>& B, int grid, cudaStream_t s);

// Pure SpMV (out = M v) over a schedule, used by the autotuner and power
// iteration.  T = float or double.
template <typename T>
void launch_spmv(const SchedView& S, const int32_t* rp, const int32_t* col, const T* val,
                 const T* v, T* out, const Launch& L, cudaStream_t s);

// float64 report of an iterate (x~, y~ given in float64):
//   part n: z, x outputs and partials [grid][4] = {U2, S3, XZ, inf_rd}
//   part m: y output and partials [grid][4] = {U1, S4, 0, inf_rp}
void launch_report_n(const SchedView& S, const int32_t* rp, const int32_t* col, const double* val,
                     const double* x_s, const double* y_s, const double* c_t, const double* D_c,
                     double* x_out, double* z_out, double* partials, const Launch& L, cudaStream_t s);
void launch_report_m(const SchedView& S, const int32_t* rp, const int32_t* col, const double* val,
                     const double* x_s, const double* y_s, const double* b_t, const double* D_r,
                     double* y_out, double* partials, const Launch& L, cudaStream_t s);
// sums the two partial sets into out[8] = {r_P, r_D, gap, maxviol, c^T x, b^T y, x^T z, 0}
void launch_report_final(const double* pn, int gn, const double* pm, int gm, double* out,
                         cudaStream_t s);

// Float64 check of a float32-mixed candidate whose screen passed (four
// launches; each returns at once unless a check is pending): the float64
// schedules and values of both matrices, conversion buffers and grids.
struct Fp64Check {
  SchedView St, Sa;            // float64 schedules of A~^T and A~
  const double *t_val, *a_val;  // float64 scaled values
  double *xs, *ys;             // candidate in float64 [n], [m]
  Launch Lt, La;
  int gn, gm;                  // block partials + split records of each report
  int conv_grid;
};
template <typename T>
void launch_fp64_check(const IterBuffers<T>& B, const Fp64Check& C, cudaStream_t s);
constexpr int kFp64CheckLaunches = 4;

// Algorithm 1 (Section 3.1)
void launch_ws_z(const SchedView& S, const int32_t* rp, const int32_t* col, const double* val,
                 const double* x_s, const double* y_s, const double* c_t, double* z_s,
                 double* partials, const Launch& L, cudaStream_t s);
void launch_ws_mu(const double* partials, int g, int n, double mu_min, double* mu, cudaStream_t s);
void launch_ws_apply(int n, int m, const double* x_s, const double* z_s, const double* y_s,
                     const double* mu, double delta_max, double alpha_min, int unscaled,
                     const double* D_r, const double* D_c, double* x_out, double* y_out,
                     double* z_out, cudaStream_t s);

// conversions and elementwise helpers
void launch_convert_d2f(const double* src, float* dst, int64_t len, cudaStream_t s);
void launch_convert_f2d(const float* src, double* dst, int64_t len, cudaStream_t s);

// ---- setup (setup_kernels.cu) -------------------------------------------
void launch_validate(int m, int n, const int32_t* rp, const int32_t* col, const double* val,
                     const double* b, const double* c, int32_t* flags, cudaStream_t s);
void launch_col_hist(int64_t nnz, const int32_t* col, int32_t* cnt, cudaStream_t s);
// exclusive scan of cnt[len] into out[len+1]; tmp holds >= len/1024 + 2 ints
void launch_scan(const int32_t* cnt, int32_t* out, int len, int32_t* tmp, cudaStream_t s);
void launch_scatter(int m, const int32_t* rp, const int32_t* col, const double* val,
                    int32_t* cursor, int32_t* col_t, double* val_t, cudaStream_t s);
void launch_segsort(int nseg, const int32_t* seg_ptr, int32_t* keys, double* vals,
                    const int32_t* long_ids, int n_long, int32_t* tmp_k, double* tmp_v,
                    cudaStream_t s);
// window words of the whole-row tiles of a segmented schedule (e = 8, 16 or
// 32 nonzeros per thread; 64-bit words for 32) over the matrix with device
// row pointer rp
void launch_window_words(const Tile* tiles, int ntiles, const int32_t* rp, int e, uint32_t* wd,
                         cudaStream_t s);
// How a row statistic pass is split: `lanes` per row (4..32, from the mean
// row length) and the rows longer than long_len (device ids), one block each.
struct RowStatPlan {
  int lanes = 32;
  int long_len = 1 << 30;
  const int32_t* long_ids = nullptr;
  int nlong = 0;
};
// Ruiz / Pock-Chambolle statistic of each row of D_self M D_other:
// mode 0: sqrt(max |.|), mode 1: sqrt(sum |.|); zero -> 1.
void launch_row_stat(int nrows, const int32_t* rp, const int32_t* col, const double* val,
                     const double* d_self, const double* d_other, int mode, double* out,
                     const RowStatPlan& plan, cudaStream_t s);
void launch_div(double* d, const double* r, int len, cudaStream_t s);
// out[i] = 1 / in[i]
void launch_recip(const double* in, double* out, int64_t len, cudaStream_t s);
void launch_fill(double* d, double v, int64_t len, cudaStream_t s);
// A~_ij = (D_r[i] A_ij) D_c[j]; transposed = 1 when the rows are columns of A
void launch_scale_vals(int nrows, const int32_t* rp, const int32_t* col, const double* val,
                       const double* D_r, const double* D_c, int transposed, double* out64,
                       float* out32, cudaStream_t s);
void launch_scale_vec(int len, const double* d, const double* v, double* out64, float* out32,
                      cudaStream_t s);
// partial sums (mode 0: a.b, 1: |a|^2, 2: |min(0,a)|^2) into partials[grid];
// then a one-thread total in fixed order
void launch_dot_partials(int64_t len, const double* a, const double* b, int mode,
                         double* partials, int grid, cudaStream_t s);
void launch_sum_final(const double* partials, int g, double* out, cudaStream_t s);
// power iteration pieces (float64)
void launch_pow_init(int n, double* v, PowerState* ps, int max_iter, double rel_tol,
                     cudaStream_t s);
void launch_pow_ATu(const SchedView& S, const int32_t* rp, const int32_t* col, const double* val,
                    const double* u, const double* v, double* w, double* partials,
                    PowerState* ps, const Launch& L, cudaStream_t s);
void launch_pow_Av(const SchedView& S, const int32_t* rp, const int32_t* col, const double* val,
                   const double* v, double* u, PowerState* ps, const Launch& L, cudaStream_t s);
void launch_pow_norm(int n, const double* w, double* v, PowerState* ps, cudaStream_t s);
// blocks per SM of the power iteration's SpMV kernels (at: the A~^T one)
int pow_occupancy(bool at, size_t smem);
// scalar set-up of the solve from reduced values
//   sums[5] = |b|^2, |c|^2, |b~|^2, |c~|^2, |min(0, c~)|^2
// eta = eta_safety / sigma_max, omega_0 = |c~|/|b~| (1 if either is 0),
// tau, sigma, and the first restart point (0, 0): kkt_last = kkt_prev =
// KKT_omega0(0, 0) = sqrt(omega^2 |b~|^2 + |min(0,c~)|^2 / omega^2)
void launch_init_scalars(Scalars* sc, const double* sums, const PowerState* ps,
                         double eta_safety, cudaStream_t s);
cudaError_t configure_setup_kernels(size_t max_smem);
// gather-rate floor pass (diagnostic): nnz nonzeros in groups of 8
template <typename T>
void launch_gather_floor(const int32_t* col, const T* val, const T* v, int64_t nnz, T* sink,
                         int grid, cudaStream_t s);
cudaError_t configure_tile_kernels(size_t max_smem);
// column-panel half-steps (panel.cu, float32): the panel SpMV then the row
// pass with the primal (dual = false) or dual epilogue of the method
// (0 averaged, 1 Halpern); row_grid blocks of 256 threads for the row pass;
// `between` (optional) is recorded between the two kernels
void launch_panel_half(const IterBuffers<float>& B, const PanelView& V, bool dual, int method,
                       int row_grid, int i, cudaStream_t s, cudaEvent_t between = nullptr);
size_t panel_smem(int P, int pscap);
// the panel SpMV kernel of a half-step alone (timing)
void launch_panel_spmv_only(const IterBuffers<float>& B, const PanelView& V, bool dual, int method,
                            cudaStream_t s);
// blocks of 256 threads for the row pass over `rows` rows of `npanels` panels
int panel_row_grid(int rows, int npanels, int nsm);
cudaError_t configure_panel_kernels(size_t max_smem);
int tile_occupancy(int which, int e, size_t smem);

// ---- reflected Halpern half-steps (halpern.cu) ----------------------------
template <typename T>
void launch_hprimal(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s);
template <typename T>
void launch_hdual(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s);
cudaError_t configure_halpern_kernels(size_t max_smem);
// blocks per SM (which: 0/1 primal f32/f64, 2/3 dual f32/f64)
int halpern_occupancy(int which, int e, size_t smem);
size_t tile_smem(int nv, bool f32, int max_rows, int e);

// ---- adaptive step (adaptive.cu) ------------------------------------------
// attempt i of the chunk: the primal half-step saving the accepted state, the
// dual half-step with the acceptance test of the attempt, and the undo of a rejected one
template <typename T>
void launch_adapt_primal(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s);
template <typename T>
void launch_adapt_dual(const IterBuffers<T>& B, const Launch& L, int i, cudaStream_t s);
template <typename T>
void launch_adapt_revert(const IterBuffers<T>& B, int grid, cudaStream_t s);
cudaError_t configure_adaptive_kernels(size_t max_smem);
// blocks per SM (which: 0/1 primal f32/f64, 2/3 dual f32/f64)
int adaptive_occupancy(int which, int e, size_t smem);

}  // namespace pdhg
