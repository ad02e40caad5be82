// L-BFGS on the angles, on the device (the paper trains QAOA angles with L-BFGS driven by
// the adjoint gradient, Sec. IV-D / V-B).  Maximising E = <C> is minimising f = -E.
//
// The optimiser is a state machine advanced once per gradient evaluation, so one
// evaluation plus one step of the machine form a fixed launch sequence that a CUDA graph
// can replay.  The evaluation point is always the angle buffer; after each evaluation:
//   * the first evaluation sets x_0 and takes the direction d = -g / max(1, |g|);
//   * otherwise the point x_k + alpha d is a line-search trial: it is accepted when the
//     Armijo condition f <= f_k + c1 alpha g_k.d holds; the pair (s, y) = (x - x_k, g - g_k)
//     enters the history when s.y > 0, and the next direction is the two-loop recursion
//     d = -H g with H_0 = s.y / y.y of the newest pair (steepest descent if that is not a
//     descent direction); a rejected trial shrinks alpha by the minimiser of the quadratic
//     through f_k, g_k.d and the trial value, kept within [0.1, 0.5] alpha;
//   * |g|_inf < gtol ends the run (converged), alpha < 1e-12 ends it (no progress).
// State (doubles): scal[16] | x | g | d | S (m rows) | Y (m rows) | rho (m).
#include "internal.h"

#include <cuda_runtime.h>

namespace qaoa {
namespace {

constexpr int kLbThreads = 128;  // >= 2p for p <= QAOA_MAX_P

enum { SC_F = 0, SC_ALPHA, SC_GTD, SC_EVALS, SC_ITERS, SC_COUNT, SC_HEAD, SC_DONE };

__device__ double block_sum(double v, double* red) {
  const int i = threadIdx.x;
  __syncthreads();
  red[i] = v;
  __syncthreads();
  for (int s = kLbThreads / 2; s > 0; s >>= 1) {
    if (i < s) red[i] += red[i + s];
    __syncthreads();
  }
  return red[0];
}
__device__ double block_max(double v, double* red) {
  const int i = threadIdx.x;
  __syncthreads();
  red[i] = v;
  __syncthreads();
  for (int s = kLbThreads / 2; s > 0; s >>= 1) {
    if (i < s) red[i] = fmax(red[i], red[i + s]);
    __syncthreads();
  }
  return red[0];
}

__global__ void __launch_bounds__(kLbThreads) lbfgs_kernel(double* __restrict__ ang, const double* __restrict__ gout,
                                                           double* __restrict__ st, int p, int m, double gtol,
                                                           double c1, double* __restrict__ history,
                                                           long long row0, long long max_rows) {
  __shared__ double red[kLbThreads];
  __shared__ double al[QAOA_LBFGS_MAX_M];
  const int i = threadIdx.x, np2 = 2 * p;
  const bool on = i < np2;
  double* scal = st;
  double* x = st + 16;
  double* g = x + np2;
  double* d = g + np2;
  double* S = d + np2;
  double* Y = S + (size_t)m * np2;
  double* rho = Y + (size_t)m * np2;
  // uniform scalars, read before anything is written
  const double fk = scal[SC_F], alpha = scal[SC_ALPHA], gtd = scal[SC_GTD];
  const long long ev = (long long)scal[SC_EVALS];
  int count = (int)scal[SC_COUNT], head = (int)scal[SC_HEAD];
  const int done = (int)scal[SC_DONE];
  if (history != nullptr && ev >= row0 && ev - row0 < max_rows && done == 0) {
    double* h = history + (ev - row0) * (2 * np2 + 2);
    for (int k = i; k < np2 + 2; k += kLbThreads) h[k] = gout[k];
    if (on) h[np2 + 2 + i] = ang[i];
  }
  if (done != 0) {  // finished: keep the evaluation point at the best accepted angles
    if (on) ang[i] = x[i];
    return;
  }
  const double ft = -gout[0];
  const double gi = on ? -gout[2 + i] : 0.0;
  const double xt = on ? ang[i] : 0.0;
  const bool accept = ev == 0 || ft <= fk + c1 * alpha * gtd;
  double new_alpha = 1.0, new_gtd = gtd, new_f = fk;
  int new_done = 0, iters_inc = 0;
  if (accept) {
    if (ev > 0) {
      const double si = on ? xt - x[i] : 0.0, yi = on ? gi - g[i] : 0.0;
      const double sy = block_sum(si * yi, red), ss = block_sum(si * si, red), yy = block_sum(yi * yi, red);
      if (sy > 1e-12 * sqrt(ss * yy) && sy > 0.0) {
        int slot;
        if (count < m) {
          slot = (head + count) % m;
          ++count;
        } else {
          slot = head;
          head = (head + 1) % m;
        }
        if (on) {
          S[(size_t)slot * np2 + i] = si;
          Y[(size_t)slot * np2 + i] = yi;
        }
        if (i == 0) rho[slot] = 1.0 / sy;
      }
      iters_inc = 1;
    }
    if (on) {
      x[i] = xt;
      g[i] = gi;
    }
    new_f = ft;
    const double ginf = block_max(on ? fabs(gi) : 0.0, red);
    if (ginf < gtol) {
      new_done = 1;
    } else {
      // two-loop recursion on q = g
      __syncthreads();  // rho written by thread 0 above
      double q = gi;
      for (int k = count - 1; k >= 0; --k) {
        const int j = (head + k) % m;
        const double a = rho[j] * block_sum(on ? S[(size_t)j * np2 + i] * q : 0.0, red);
        if (i == 0) al[k] = a;
        if (on) q -= a * Y[(size_t)j * np2 + i];
      }
      double h0;
      if (count > 0) {
        const int j = (head + count - 1) % m;
        const double yj = on ? Y[(size_t)j * np2 + i] : 0.0;
        h0 = 1.0 / (rho[j] * block_sum(yj * yj, red));
      } else {
        h0 = 1.0 / fmax(1.0, sqrt(block_sum(gi * gi, red)));
      }
      double r = h0 * q;
      __syncthreads();  // al visible
      for (int k = 0; k < count; ++k) {
        const int j = (head + k) % m;
        const double b = rho[j] * block_sum(on ? Y[(size_t)j * np2 + i] * r : 0.0, red);
        if (on) r += S[(size_t)j * np2 + i] * (al[k] - b);
      }
      double di = -r;
      double gd = block_sum(on ? gi * di : 0.0, red);
      if (!(gd < 0.0)) {  // not a descent direction: restart from steepest descent
        count = 0;
        head = 0;
        di = -gi / fmax(1.0, sqrt(block_sum(gi * gi, red)));
        gd = block_sum(on ? gi * di : 0.0, red);
      }
      if (on) d[i] = di;
      new_gtd = gd;
      new_alpha = 1.0;
    }
  } else {
    // safeguarded quadratic backtracking
    const double den = 2.0 * (ft - fk - gtd * alpha);
    double a = den > 0.0 ? -gtd * alpha * alpha / den : 0.5 * alpha;
    a = fmin(fmax(a, 0.1 * alpha), 0.5 * alpha);
    new_alpha = a;
    if (a < 1e-12) new_done = 2;
  }
  __syncthreads();
  if (on) ang[i] = new_done ? x[i] : fma(new_alpha, d[i], x[i]);  // the resume kernel rounds the same way
  if (i == 0) {
    scal[SC_F] = new_f;
    scal[SC_ALPHA] = new_alpha;
    scal[SC_GTD] = new_gtd;
    scal[SC_EVALS] = (double)(ev + 1);
    scal[SC_ITERS] += iters_inc;
    scal[SC_COUNT] = count;
    scal[SC_HEAD] = head;
    scal[SC_DONE] = new_done;
  }
}

// resuming: the evaluation point goes back to the trial the state machine expects next
__global__ void lbfgs_resume_kernel(double* __restrict__ ang, const double* __restrict__ st, int p) {
  const int i = threadIdx.x;
  if (i < 2 * p && st[SC_EVALS] > 0 && st[SC_DONE] == 0) {
    const double* x = st + 16;
    ang[i] = fma(st[SC_ALPHA], x[4 * p + i], x[i]);  // d follows x and g
  }
}

// after the last evaluation: the angles go to the best accepted point; info = [E at it,
// accepted iterations, evaluations, status (0 running out of evaluations, 1 converged,
// 2 no progress)]
__global__ void lbfgs_finish_kernel(double* __restrict__ ang, const double* __restrict__ st, int p,
                                    double* __restrict__ info) {
  const int i = threadIdx.x;
  if (i < 2 * p && st[SC_EVALS] > 0) ang[i] = st[16 + i];
  if (i == 0 && info != nullptr) {
    info[0] = -st[SC_F];
    info[1] = st[SC_ITERS];
    info[2] = st[SC_EVALS];
    info[3] = st[SC_DONE];
  }
}

}  // namespace

size_t lbfgs_state_doubles(int p, int m) { return 16 + 3 * (size_t)(2 * p) + 2 * (size_t)m * 2 * p + m; }

cudaError_t launch_lbfgs(double* ang, const double* gout, double* st, int p, int m, double gtol, double c1,
                         double* history, long long row0, long long max_rows, cudaStream_t s) {
  note_launch(3, s, true);
  lbfgs_kernel<<<1, kLbThreads, 0, s>>>(ang, gout, st, p, m, gtol, c1, history, row0, max_rows);
  note_launch(3, s, false);
  return cudaGetLastError();
}

cudaError_t launch_lbfgs_resume(double* ang, const double* st, int p, cudaStream_t s) {
  note_launch(3, s, true);
  lbfgs_resume_kernel<<<1, kLbThreads, 0, s>>>(ang, st, p);
  note_launch(3, s, false);
  return cudaGetLastError();
}

cudaError_t launch_lbfgs_finish(double* ang, const double* st, int p, double* info, cudaStream_t s) {
  note_launch(3, s, true);
  lbfgs_finish_kernel<<<1, kLbThreads, 0, s>>>(ang, st, p, info);
  note_launch(3, s, false);
  return cudaGetLastError();
}

}  // namespace qaoa
