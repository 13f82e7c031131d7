// Row epilogues of the PDHG half-steps: given row r's product s (a row of
// A~^T y for the primal, of A~ x for the dual), update that row's iterate and
// caches.  Shared by the fused CSR tile kernels (the epilogue runs as each tile
// finishes its rows) and the column-panel path (a separate pass after the
// panel partial sums are added).  Each epilogue reads its row's operands
// with load(i) and writes with apply(i, in, s): the panel row pass issues
// load(i) before the partial sums arrive; row() is the two in sequence.
#pragma once

namespace pdhg {

// K1: x+ = max(0, x - tau (c~ - A~^T y)), running average of x.
template <typename T>
struct PrimalEpi {
  T* __restrict__ x;
  const T* __restrict__ c;
  T* __restrict__ x_avg;
  T tau, w;
  bool first;
  struct In {
    T x, c, xa;
  };
  __device__ __forceinline__ In load(int j) const {
    return In{x[j], c[j], first ? T(0) : x_avg[j]};
  }
  __device__ __forceinline__ void apply(int j, const In& in, T s) {
    const T xn = fmax(T(0), in.x - tau * (in.c - s));
    x[j] = xn;
    x_avg[j] = first ? xn : in.xa + (xn - in.xa) * w;
  }
  __device__ __forceinline__ void row(int j, const T (&s)[1], int) { apply(j, load(j), s[0]); }
};

// K2: h = A~ x+;  y+ = y + sigma (b~ - 2h + A~x)   (= b~ - A~(2x+ - x));
// caches A~x+ and the running averages of y and A~x.
template <typename T>
struct DualEpi {
  T* __restrict__ y;
  const T* __restrict__ b;
  T* __restrict__ Ax;
  T* __restrict__ y_avg;
  T* __restrict__ Ax_avg;
  T sigma, w;
  bool first;
  struct In {
    T y, b, ax, ya, axa;
  };
  __device__ __forceinline__ In load(int i) const {
    return In{y[i], b[i], Ax[i], first ? T(0) : y_avg[i], first ? T(0) : Ax_avg[i]};
  }
  __device__ __forceinline__ void apply(int i, const In& in, T h) {
    const T yn = in.y + sigma * (in.b - (h + h) + in.ax);
    Ax[i] = h;
    y[i] = yn;
    y_avg[i] = first ? yn : in.ya + (yn - in.ya) * w;
    Ax_avg[i] = first ? h : in.axa + (h - in.axa) * w;
  }
  __device__ __forceinline__ void row(int i, const T (&s)[1], int) { apply(i, load(i), s[0]); }
};

// Reflected Halpern iteration, primal: x^ = T(z)_x into x_hat, the new x in
// place (lam = (t+1)/(t+2), anchor x0).
template <typename T>
struct HalpernPrimalEpi {
  T* __restrict__ x;
  T* __restrict__ x_hat;
  const T* __restrict__ c;
  const T* __restrict__ x0;
  T tau, lam, rho;
  struct In {
    T xo, c, x0;
  };
  __device__ __forceinline__ In load(int j) const { return In{x[j], c[j], x0[j]}; }
  __device__ __forceinline__ void apply(int j, const In& in, T s) {
    const T xh = fmax(T(0), in.xo - tau * (in.c - s));
    x_hat[j] = xh;
    x[j] = lam * ((T(1) + rho) * xh - rho * in.xo) + (T(1) - lam) * in.x0;
  }
  __device__ __forceinline__ void row(int j, const T (&s)[1], int) { apply(j, load(j), s[0]); }
};

// Reflected Halpern iteration, dual: y^ into y_hat, h into Ax_hat, the new y
// and the cache A~x by linearity.
template <typename T>
struct HalpernDualEpi {
  T* __restrict__ y;
  const T* __restrict__ b;
  T* __restrict__ Ax;
  T* __restrict__ y_hat;
  T* __restrict__ Ax_hat;
  const T* __restrict__ y0;
  const T* __restrict__ Ax0;
  T sigma, lam, rho;
  struct In {
    T yo, b, axo, y0, ax0;
  };
  __device__ __forceinline__ In load(int i) const {
    return In{y[i], b[i], Ax[i], y0[i], Ax0[i]};
  }
  __device__ __forceinline__ void apply(int i, const In& in, T h) {
    const T yh = in.yo + sigma * (in.b - (h + h) + in.axo);
    y_hat[i] = yh;
    Ax_hat[i] = h;
    y[i] = lam * ((T(1) + rho) * yh - rho * in.yo) + (T(1) - lam) * in.y0;
    Ax[i] = lam * ((T(1) + rho) * h - rho * in.axo) + (T(1) - lam) * in.ax0;
  }
  __device__ __forceinline__ void row(int i, const T (&s)[1], int) { apply(i, load(i), s[0]); }
};

}  // namespace pdhg
