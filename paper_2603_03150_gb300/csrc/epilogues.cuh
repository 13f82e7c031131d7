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
  // four consecutive rows j..j+3 (j a multiple of 4; float only)
  struct In4 {
    float4 x, c, xa;
  };
  __device__ __forceinline__ In4 load4(int j) const {
    In4 r;
    r.x = *reinterpret_cast<const float4*>(x + j);
    r.c = *reinterpret_cast<const float4*>(c + j);
    r.xa = first ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(x_avg + j);
    return r;
  }
  __device__ __forceinline__ void apply4(int j, const In4& in, const float4& s) {
    const float4 xn = make_float4(fmaxf(0.f, in.x.x - tau * (in.c.x - s.x)),
                                  fmaxf(0.f, in.x.y - tau * (in.c.y - s.y)),
                                  fmaxf(0.f, in.x.z - tau * (in.c.z - s.z)),
                                  fmaxf(0.f, in.x.w - tau * (in.c.w - s.w)));
    *reinterpret_cast<float4*>(x + j) = xn;
    *reinterpret_cast<float4*>(x_avg + j) =
        first ? xn
              : make_float4(in.xa.x + (xn.x - in.xa.x) * w, in.xa.y + (xn.y - in.xa.y) * w,
                            in.xa.z + (xn.z - in.xa.z) * w, in.xa.w + (xn.w - in.xa.w) * w);
  }
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
  struct In4 {
    float4 y, b, ax, ya, axa;
  };
  __device__ __forceinline__ In4 load4(int i) const {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    In4 r;
    r.y = *reinterpret_cast<const float4*>(y + i);
    r.b = *reinterpret_cast<const float4*>(b + i);
    r.ax = *reinterpret_cast<const float4*>(Ax + i);
    r.ya = first ? z : *reinterpret_cast<const float4*>(y_avg + i);
    r.axa = first ? z : *reinterpret_cast<const float4*>(Ax_avg + i);
    return r;
  }
  __device__ __forceinline__ void apply4(int i, const In4& in, const float4& h) {
    const float4 yn = make_float4(in.y.x + sigma * (in.b.x - (h.x + h.x) + in.ax.x),
                                  in.y.y + sigma * (in.b.y - (h.y + h.y) + in.ax.y),
                                  in.y.z + sigma * (in.b.z - (h.z + h.z) + in.ax.z),
                                  in.y.w + sigma * (in.b.w - (h.w + h.w) + in.ax.w));
    *reinterpret_cast<float4*>(Ax + i) = h;
    *reinterpret_cast<float4*>(y + i) = yn;
    *reinterpret_cast<float4*>(y_avg + i) =
        first ? yn
              : make_float4(in.ya.x + (yn.x - in.ya.x) * w, in.ya.y + (yn.y - in.ya.y) * w,
                            in.ya.z + (yn.z - in.ya.z) * w, in.ya.w + (yn.w - in.ya.w) * w);
    *reinterpret_cast<float4*>(Ax_avg + i) =
        first ? h
              : make_float4(in.axa.x + (h.x - in.axa.x) * w, in.axa.y + (h.y - in.axa.y) * w,
                            in.axa.z + (h.z - in.axa.z) * w, in.axa.w + (h.w - in.axa.w) * w);
  }
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
  struct In4 {
    float4 xo, c, x0;
  };
  __device__ __forceinline__ In4 load4(int j) const {
    return In4{*reinterpret_cast<const float4*>(x + j), *reinterpret_cast<const float4*>(c + j),
               *reinterpret_cast<const float4*>(x0 + j)};
  }
  __device__ __forceinline__ float one(float xo, float cc, float x0v, float s, float* xh) const {
    *xh = fmaxf(0.f, xo - tau * (cc - s));
    return lam * ((1.f + rho) * *xh - rho * xo) + (1.f - lam) * x0v;
  }
  __device__ __forceinline__ void apply4(int j, const In4& in, const float4& s) {
    float4 xh, xn;
    xn.x = one(in.xo.x, in.c.x, in.x0.x, s.x, &xh.x);
    xn.y = one(in.xo.y, in.c.y, in.x0.y, s.y, &xh.y);
    xn.z = one(in.xo.z, in.c.z, in.x0.z, s.z, &xh.z);
    xn.w = one(in.xo.w, in.c.w, in.x0.w, s.w, &xh.w);
    *reinterpret_cast<float4*>(x_hat + j) = xh;
    *reinterpret_cast<float4*>(x + j) = xn;
  }
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
  struct In4 {
    float4 yo, b, axo, y0, ax0;
  };
  __device__ __forceinline__ In4 load4(int i) const {
    return In4{*reinterpret_cast<const float4*>(y + i), *reinterpret_cast<const float4*>(b + i),
               *reinterpret_cast<const float4*>(Ax + i), *reinterpret_cast<const float4*>(y0 + i),
               *reinterpret_cast<const float4*>(Ax0 + i)};
  }
  __device__ __forceinline__ void one(float yo, float bb, float axo, float y0v, float ax0v, float h,
                                      float* yh, float* yn, float* axn) const {
    *yh = yo + sigma * (bb - (h + h) + axo);
    *yn = lam * ((1.f + rho) * *yh - rho * yo) + (1.f - lam) * y0v;
    *axn = lam * ((1.f + rho) * h - rho * axo) + (1.f - lam) * ax0v;
  }
  __device__ __forceinline__ void apply4(int i, const In4& in, const float4& h) {
    float4 yh, yn, axn;
    one(in.yo.x, in.b.x, in.axo.x, in.y0.x, in.ax0.x, h.x, &yh.x, &yn.x, &axn.x);
    one(in.yo.y, in.b.y, in.axo.y, in.y0.y, in.ax0.y, h.y, &yh.y, &yn.y, &axn.y);
    one(in.yo.z, in.b.z, in.axo.z, in.y0.z, in.ax0.z, h.z, &yh.z, &yn.z, &axn.z);
    one(in.yo.w, in.b.w, in.axo.w, in.y0.w, in.ax0.w, h.w, &yh.w, &yn.w, &axn.w);
    *reinterpret_cast<float4*>(y_hat + i) = yh;
    *reinterpret_cast<float4*>(Ax_hat + i) = h;
    *reinterpret_cast<float4*>(y + i) = yn;
    *reinterpret_cast<float4*>(Ax + i) = axn;
  }
};

}  // namespace pdhg
