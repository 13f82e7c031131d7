// The on-device termination test (Section 2) and restart rule, shared by the
// single-LP and batched evaluation kernels.
#pragma once
#include <math.h>

#include "common.cuh"

namespace pdhg {

__device__ __forceinline__ bool finite3(double a, double b, double c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}

// Termination test (Section 2) for one LP after `chunk` more iterations, from
// the reduced sums tot[2][Q_N] (current, average).  True when the evaluation
// is decided: converged, a non-finite value, the iteration limit, or (with
// fp64_check) a screen pass that a float64 check must confirm.  Runs in one
// thread.
__device__ inline bool eval_termination(Scalars& sc, const double* tot, int chunk) {
  sc.k += chunk;
  sc.t += chunk;
  for (int c = 0; c < 2; ++c)
    for (int k = 0; k < Q_N; ++k) sc.q[c][k] = tot[c * Q_N + k];
  const double eps = sc.fp64_check ? sc.eps * sc.screen : sc.eps;
  bool term[2];
  bool bad = false;
  for (int c = 0; c < 2; ++c) {
    const double* q = tot + c * Q_N;
    const double rp = sqrt(q[Q_U1]), rd = sqrt(q[Q_U2]);
    const double pobj = q[Q_S3], dobj = q[Q_S4];
    if (!finite3(rp, rd, pobj - dobj)) bad = true;
    term[c] = rp <= eps * (1.0 + sc.norm_b) && rd <= eps * (1.0 + sc.norm_c) &&
              fabs(pobj - dobj) <= eps * (1.0 + fabs(pobj) + fabs(dobj));
  }
  sc.restart_pending = 0;
  if (term[0] || term[1]) {
    if (sc.fp64_check) {
      sc.verify = 1;
      sc.verify_avg = term[0] ? 0 : 1;
      sc.checks += 1;
      return true;
    }
    sc.done = 1;
    sc.status = 0;
    sc.chosen_avg = term[0] ? 0 : 1;
    return true;
  }
  if (bad) {
    sc.done = 1;
    sc.status = 2;
    sc.chosen_avg = 0;
    return true;
  }
  if (sc.k >= sc.max_iter) {
    sc.done = 1;
    sc.status = 1;
    sc.chosen_avg = 0;
    return true;
  }
  return false;
}

// The restart rule and primal-weight update at an evaluation with k % F == 0,
// from the reduced sums tot[2][Q_N].  The log pointers may be NULL (no log).
__device__ inline void eval_restart(Scalars& sc, const double* tot, long long* log_k,
                                    int32_t* log_flags, double* log_kkt) {
  if (sc.k % sc.eval_freq != 0) return;
  const double w2 = sc.omega * sc.omega;
  double kkt[2];
  for (int c = 0; c < 2; ++c) {
    const double* q = tot + c * Q_N;
    const double gap = q[Q_S3] - q[Q_S4];
    kkt[c] = sqrt(w2 * q[Q_S1] + q[Q_S2] / w2 + gap * gap);
  }
  const int cand = (kkt[1] < kkt[0]) ? 1 : 0;
  const double kc = kkt[cand];
  const bool r1 = kc <= sc.beta_suff * sc.kkt_last;
  const bool r2 = (kc <= sc.beta_nec * sc.kkt_last) && (kc > sc.kkt_prev);
  const bool r3 = (double)sc.t >= sc.beta_art * (double)sc.k;
  const bool restart = r1 || r2 || r3;
  if (log_k && sc.log_count < sc.log_cap) {
    const int e = sc.log_count++;
    log_k[e] = sc.k;
    log_flags[e] = (restart ? 1 : 0) | (cand << 1) | (r1 << 2) | (r2 << 3) | (r3 << 4);
    log_kkt[3 * e + 0] = kkt[0];
    log_kkt[3 * e + 1] = kkt[1];
    log_kkt[3 * e + 2] = sc.omega;
  }
  sc.kkt_prev = kc;
  if (restart) {
    const double dx = sqrt(tot[cand * Q_N + Q_D1]);
    const double dy = sqrt(tot[cand * Q_N + Q_D2]);
    if (dx > 1e-10 && dy > 1e-10) {
      if (sc.omega_rule == 1) {
        // PID control of log omega: e = log(dy/dx) - log omega, I += e
        const double e = log(dy / dx) - log(sc.omega);
        sc.pid_integral += e;
        sc.omega = exp(log(sc.omega) + sc.pid_kp * e + sc.pid_ki * sc.pid_integral +
                       sc.pid_kd * (e - sc.pid_prev));
        sc.pid_prev = e;
      } else {
        sc.omega = exp(sc.theta * log(dy / dx) + (1.0 - sc.theta) * log(sc.omega));
      }
    }
    sc.tau = sc.eta / sc.omega;
    sc.sigma = sc.eta * sc.omega;
    sc.t = 0;
    if (sc.step_rule) {  // the step-weighted averages restart too
      sc.eta_sum = 0.0;
      sc.avg_w = 1.0;
      sc.avg_first = 1;
    }
    sc.restarts += 1;
    sc.kkt_last = kc;
    sc.restart_pending = 1;
    sc.restart_to_avg = cand;
  }
}

// Termination test, then (if undecided) the restart rule.
__device__ inline void apply_eval_rule(Scalars& sc, const double* tot, int chunk, long long* log_k,
                                       int32_t* log_flags, double* log_kkt) {
  if (eval_termination(sc, tot, chunk)) return;
  eval_restart(sc, tot, log_k, log_flags, log_kkt);
}

// The float64 check of a screened candidate: sums = {||r_P||^2, ||r_D||^2,
// c^T x, b^T y} of the candidate in the original model, every product
// recomputed in float64.  It passes the Section 2 test at eps itself: the
// solve ends with that candidate.  Otherwise the evaluation continues where
// the screen stopped it (the iteration limit, then the restart rule on the
// evaluation's stored sums).
__device__ inline void eval_fp64_check(Scalars& sc, double u1, double u2, double s3, double s4,
                                       long long* log_k, int32_t* log_flags, double* log_kkt) {
  sc.verify = 0;
  const double rp = sqrt(u1), rd = sqrt(u2), gap = fabs(s3 - s4);
  const bool ok = rp <= sc.eps * (1.0 + sc.norm_b) && rd <= sc.eps * (1.0 + sc.norm_c) &&
                  gap <= sc.eps * (1.0 + fabs(s3) + fabs(s4));
  if (ok) {
    sc.done = 1;
    sc.status = 0;
    sc.chosen_avg = sc.verify_avg;
    return;
  }
  sc.rejects += 1;
  if (sc.k >= sc.max_iter) {
    sc.done = 1;
    sc.status = 1;
    sc.chosen_avg = 0;
    return;
  }
  eval_restart(sc, &sc.q[0][0], log_k, log_flags, log_kkt);
}

}  // namespace pdhg
