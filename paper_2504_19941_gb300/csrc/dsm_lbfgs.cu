// dsm_lbfgs.cu -- the energy minimiser's L-BFGS loop, run natively on the host
// around the library's kernels (Sec. II.A of the paper minimises the discrete
// free energy with L-BFGS, citing Nocedal 1980 and Liu & Nocedal 1989, with an
// rms-gradient stop; it fixes neither the history length nor the line search).
//
// Readings: m pairs (caller's choice, 10 by default in the binding),
// H0 = (s.y / y.y) I, pairs with s.y <= 1e-12 |s||y| dropped, strong-Wolfe
// line search (c1 = 1e-4, c2 = 0.9) that brackets and then shrinks the bracket
// with a safeguarded cubic, at most 20 trials.  Near FP32 noise the
// sufficient-decrease test uses its derivative form (the approximate Wolfe
// condition of Hager & Zhang 2005).  The direction comes from the compact form
// of the L-BFGS matrix (Byrd, Nocedal & Schnabel 1994), the matrix the
// two-loop recursion applies: one batched pass of dot products over the pairs
// and one linear combination per iteration.
//
// The pair bookkeeping (the s.y and y.y matrices, S^T g, Y^T g, gamma, the
// ring of stored pairs) and the compact-form solve live on the device, in one
// small state block updated by one-thread kernels; the host drives only the
// line search, whose decisions need the trial's energy and slope.  Each trial
// reads one block of six doubles (slope, energy, the direction's initial
// slope, |g|^2 of the current point, the pairs in use, the next pair's slot),
// so an iteration whose first trial is accepted reads the host once.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dsm_em.cuh"
#include "dsm_trace.cuh"

using namespace dsm;

constexpr int LB_MAX_M = LINCOMB_MAX / 2;  // most stored pairs

namespace {

// Compact-form coefficients: R w = a, R^T u = (D + gamma YY) w - gamma b,
// d = -gamma g - S u + gamma Y w.  Pair i (oldest first) is stored in slot
// ord[i] of m: s_i.y_j = SY[ord[i] m + ord[j]], y_i.y_j likewise in YY,
// a_i = A[ord[i]], b_i = B[ord[i]]; R is the upper triangle of (s_i.y_j), D its
// diagonal.  w, z, u: k reals of scratch.  (The device's solve, in
// lb_step_kernel, is the same algebra spread over a warp.)
bool compact_slots(int k, const int *ord, int m, const double *SY,
                                       const double *YY, const double *A, const double *B,
                                       double gamma, double *w, double *z, double *u, double *cx,
                                       double *cs, double *cy) {
  for (int i = k - 1; i >= 0; i--) {  // back substitution, R upper triangular
    double v = A[ord[i]];
    for (int j = i + 1; j < k; j++) v -= SY[ord[i] * m + ord[j]] * w[j];
    const double d = SY[ord[i] * m + ord[i]];
    if (!(d != 0.0)) return false;
    w[i] = v / d;
  }
  for (int i = 0; i < k; i++) {
    double v = SY[ord[i] * m + ord[i]] * w[i] - gamma * B[ord[i]];
    for (int j = 0; j < k; j++) v += gamma * YY[ord[i] * m + ord[j]] * w[j];
    z[i] = v;
  }
  for (int i = 0; i < k; i++) {  // forward substitution, R^T lower triangular
    double v = z[i];
    for (int j = 0; j < i; j++) v -= SY[ord[j] * m + ord[i]] * u[j];
    u[i] = v / SY[ord[i] * m + ord[i]];
  }
  *cx = -gamma;
  for (int i = 0; i < k; i++) {
    cs[i] = -u[i];
    cy[i] = gamma * w[i];
  }
  return true;
}

// The minimiser's state on the device.  rb: the block each trial reads back
// (slope of the trial, its energy, initial slope dg0 of the direction, |g|^2
// of the current point, pairs in use by the direction (0: steepest descent),
// slot of the next pair).
struct LbState {
  double rb[6];  // first: the host reads it at the state's address
  double gamma, cx;
  int k, nxt;
  int order[LB_MAX_M];  // slots of the stored pairs, oldest first
  double SY[LB_MAX_M * LB_MAX_M], YY[LB_MAX_M * LB_MAX_M], Ag[LB_MAX_M], Bg[LB_MAX_M];
  double coef[2 * LB_MAX_M];  // the direction: cx g + sum coef_j (s_0..s_{m-1}, y_0..y_{m-1})_j
};

__global__ void lb_init_kernel(LbState *s) {
  s->gamma = 1.0;
  s->cx = 0.0;
  s->k = 0;
  s->nxt = 0;
  for (int i = 0; i < LB_MAX_M * LB_MAX_M; i++) s->SY[i] = s->YY[i] = 0.0;
  for (int i = 0; i < LB_MAX_M; i++) s->Ag[i] = s->Bg[i] = 0.0;
  for (int i = 0; i < 2 * LB_MAX_M; i++) s->coef[i] = 0.0;
}

// One warp per iteration.  (1) If `dots` is given: the accepted step's pair
// (s, y already stored in slot nxt).  dots[i] = s_i.g and dots[m + i] = y_i.g
// for every slot against the new gradient g (slot nxt holding the new pair),
// dots[2m] = y.y, dots[2m + 1] = g.g, dots[2m + 2] = s.s; sy = s.y of the new
// pair, from the line search's slopes.  The new column of the pair matrices
// needs no pass of its own: s_i.y = s_i.g - s_i.g_old and y_i.y = y_i.g -
// y_i.g_old, where s_i.g_old and y_i.g_old are the previous iteration's
// S^T g and Y^T g (Ag, Bg).  The pair replaces the one in slot nxt (the oldest
// in a full ring) if s.y > 1e-12 |s||y|.  (2) The direction of the
// current point from the stored pairs (compact form), or steepest descent
// when there are none or the compact direction does not descend (the pairs
// are then dropped): coef, cx, and rb[2] .. rb[5].  The pairs' k x k matrices
// are staged into shared memory by the lanes and solved there by the warp.
__global__ void __launch_bounds__(32) lb_step_kernel(LbState *s, const double *dots, int m,
                                                     double sy1) {
  __shared__ double sy[LB_MAX_M * LB_MAX_M], yy[LB_MAX_M * LB_MAX_M];
  __shared__ double A[LB_MAX_M], B[LB_MAX_M], w[LB_MAX_M];
  __shared__ double cs[LB_MAX_M], cy[LB_MAX_M];
  __shared__ int ord[LB_MAX_M];
  __shared__ int ok_s;
  const int l = threadIdx.x;
  if (dots) {
    const int nxt = s->nxt;
    const double yy1 = dots[2 * m], ss = dots[2 * m + 2];
    const bool accept = sy1 > 1e-12 * sqrt(ss * yy1);
    for (int i = l; i < m; i += 32) {
      const double agn = dots[i], bgn = dots[m + i];
      if (accept) {
        if (i == nxt) {
          s->SY[i * m + nxt] = sy1;
          s->YY[i * m + nxt] = yy1;
        } else {
          const double yy_i = bgn - s->Bg[i];  // y_i . y_new
          s->SY[i * m + nxt] = agn - s->Ag[i];  // s_i . y_new
          s->YY[i * m + nxt] = yy_i;
          s->YY[nxt * m + i] = yy_i;
        }
      }
      s->Ag[i] = agn;
      s->Bg[i] = bgn;
    }
    if (l == 0) {
      int k = 0;
      for (int i = 0; i < s->k; i++)
        if (s->order[i] != nxt) s->order[k++] = s->order[i];
      if (accept) {
        s->gamma = sy1 / yy1;
        s->order[k++] = nxt;
        s->nxt = (nxt + 1) % m;
      }
      s->k = k;
      s->rb[3] = dots[2 * m + 1];
    }
    __syncthreads();
  }
  const int k = s->k;
  const double gg = s->rb[3], gamma = s->gamma;
  for (int i = l; i < k; i += 32) {
    ord[i] = s->order[i];
  }
  __syncthreads();
  for (int i = l; i < k; i += 32) {
    for (int j = 0; j < k; j++) {
      sy[i * k + j] = s->SY[ord[i] * m + ord[j]];
      yy[i * k + j] = s->YY[ord[i] * m + ord[j]];
    }
    A[i] = s->Ag[ord[i]];
    B[i] = s->Bg[ord[i]];
  }
  __syncthreads();
  // the compact-form solve across the warp (lane l owns pair l): the
  // triangular substitutions column by column with the diagonal's
  // reciprocals, the middle product row by row, dg0 by a warp reduction
  const unsigned full = 0xffffffffu;
  bool ok = k > 0;
  double cx = -gamma, dg0 = 0.0, wl = 0.0, ul = 0.0;
  if (ok) {
    const double dl = l < k ? sy[l * k + l] : 1.0;
    ok = __all_sync(full, dl != 0.0);
    if (ok) {
      const double inv = 1.0 / dl;
      double r = l < k ? A[l] : 0.0;  // R w = a, R upper triangular
      for (int i = k - 1; i >= 0; i--) {
        const double wi = __shfl_sync(full, r, i) * __shfl_sync(full, inv, i);
        if (l == i) wl = wi;
        if (l < i) r -= sy[l * k + i] * wi;
      }
      if (l < k) w[l] = wl;
      __syncwarp();
      double zl = 0.0;  // (D + gamma YY) w - gamma b
      if (l < k) {
        zl = sy[l * k + l] * wl - gamma * B[l];
        for (int j = 0; j < k; j++) zl += gamma * yy[l * k + j] * w[j];
      }
      for (int j = 0; j < k; j++) {  // R^T u = z, R^T lower triangular
        const double uj = __shfl_sync(full, zl, j) * __shfl_sync(full, inv, j);
        if (l == j) ul = uj;
        if (l > j) zl -= sy[j * k + l] * uj;
      }
      double part = l < k ? -ul * A[l] + gamma * wl * B[l] : 0.0;
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(full, part, o);
      dg0 = cx * gg + part;
      ok = dg0 < 0.0;
    }
  }
  if (!ok) {  // no pairs, or not a descent direction: steepest descent
    cx = -1.0 / fmax(sqrt(gg), 1e-300);
    dg0 = cx * gg;
  }
  if (l < k) {
    cs[l] = -ul;
    cy[l] = gamma * wl;
  }
  if (l == 0) {
    ok_s = ok;
    s->k = ok ? k : 0;
    s->cx = cx;
    s->rb[2] = dg0;
    s->rb[4] = ok ? (double)k : 0.0;
    s->rb[5] = (double)s->nxt;
  }
  __syncthreads();
  for (int i = l; i < 2 * m; i += 32) s->coef[i] = 0.0;
  __syncthreads();
  if (ok_s)
    for (int i = l; i < k; i += 32) {
      s->coef[ord[i]] = cs[i];
      s->coef[m + ord[i]] = cy[i];
    }
}

// d = cx g + sum_j coef_j V_j over the 2m stored vectors, coefficients from
// the device state (a vector with a zero coefficient is not read)
__global__ void __launch_bounds__(256) lb_lincomb_kernel(long long n, int nv, const float *V,
                                                         long long stride, const LbState *s,
                                                         const float *g, float *d) {
  __shared__ float c[2 * LB_MAX_M];
  __shared__ float cx;
  if (threadIdx.x < nv) c[threadIdx.x] = (float)s->coef[threadIdx.x];
  if (threadIdx.x == 0) cx = (float)s->cx;
  __syncthreads();
  // four elements a grid apart per iteration: four loads per stream in flight
  const long long G = (long long)gridDim.x * blockDim.x;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; k + 3 * G < n; k += 4 * G) {
    float acc[4];
#pragma unroll
    for (int u = 0; u < 4; u++) acc[u] = cx * g[k + u * G];
    for (int j = 0; j < nv; j++) {
      if (c[j] == 0.0f) continue;
      const float *vj = V + j * stride + k;
      float vv[4];
#pragma unroll
      for (int u = 0; u < 4; u++) vv[u] = vj[u * G];
#pragma unroll
      for (int u = 0; u < 4; u++) acc[u] += c[j] * vv[u];
    }
#pragma unroll
    for (int u = 0; u < 4; u++) d[k + u * G] = acc[u];
  }
  for (; k < n; k += G) {
    float acc = cx * g[k];
    for (int j = 0; j < nv; j++)
      if (c[j] != 0.0f) acc += c[j] * V[j * stride + k];
    d[k] = acc;
  }
}

// drop the stored pairs (after a line search that found no step)
__global__ void lb_reset_kernel(LbState *s) { s->k = 0; }

// Minimiser of the cubic through (a, fa, da), (b, fb, db), kept in the middle
// 80 % of the bracket (bisection otherwise).
double cubic_step(double a, double fa, double da, double b, double fb, double db) {
  const double lo = std::min(a, b), hi = std::max(a, b);
  const double den = b - a;
  double t = NAN;
  if (den != 0.0) {
    const double z = 3.0 * (fa - fb) / den + da + db;
    const double w2 = z * z - da * db;
    if (w2 >= 0.0) {
      const double w = copysign(sqrt(w2), den);
      const double q = db - da + 2.0 * w;
      if (q != 0.0) t = b - den * (db + w - z) / q;
    }
  }
  if (!(t >= lo + 0.1 * (hi - lo) && t <= hi - 0.1 * (hi - lo))) t = 0.5 * (lo + hi);
  return t;
}

struct Minimiser {
  long long n;  // vector length: nodes, or nodes x free fluids
  int m;
  cudaStream_t st;
  FEArgs fa;
  int kind;
  double dP, kcs, V0;
  const float *fixed;
  int active;
  bool multi = false;  // N fluids: x holds the free fluid planes
  FEMArgs fm;
  FEMCons fcons;
  // device buffers (carved from the caller's workspace)
  float *xb[2], *gb[2], *d, *hist;
  double *E[2], *dots, *vout;  // vout: the state's read-back block
  LbState *state;
  void *fe_scr, *vec_scr, *dots_scr;

  cudaError_t evaluate(const float *x, double *e_out, float *g_out) {
    if (multi) {
      FEMArgs b = fm;
      b.c = x;
      b.grad = g_out;
      return fe_multi_launch(kind, b, fcons, e_out, nullptr, fe_scr, st);
    }
    FEArgs a = fa;
    a.c1 = active == 2 ? fixed : x;
    a.c2 = active == 2 ? x : fixed;
    a.grad = g_out;
    return fe_launch(kind, a, dP, kcs, V0, e_out, nullptr, fe_scr, st);
  }
  // device doubles -> host (pageable copy, waits for the stream)
  cudaError_t read(double *h, const double *dv, int count) {
    cudaError_t e = cudaMemcpyAsync(h, dv, count * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  }
  // trial point xt = x + a d: energy and directional derivative, read back
  // with the rest of the state's block (rb: 6 doubles).  Two fluids: the
  // energy goes straight into the block, and the constraint's constant is
  // added to the gradient in the same pass that takes the slope.
  cudaError_t trial(double a, const float *x, float *xt, double *Et, float *gt, double *rb) {
    cudaError_t e = vec_lincomb(n, 1, d, n, &a, x, 1.0, xt, st);
    if (multi) {
      if (e == cudaSuccess) e = evaluate(xt, Et, gt);
      if (e == cudaSuccess) e = vec_dot(n, gt, d, vout, nullptr, vec_scr, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(vout + 1, Et, sizeof(double), cudaMemcpyDeviceToDevice, st);
    } else {
      FEArgs b = fa;
      b.c1 = active == 2 ? fixed : xt;
      b.c2 = active == 2 ? xt : fixed;
      b.grad = gt;
      const double *cst = nullptr;
      if (e == cudaSuccess) e = fe_launch(kind, b, dP, kcs, V0, vout + 1, nullptr, fe_scr, st, &cst);
      if (e == cudaSuccess) e = vec_trial_slope(n, cst, gt, d, vout, vec_scr, st);
    }
    if (e == cudaSuccess) e = read(rb, vout, 6);
    return e;
  }
};

}  // namespace

// The L-BFGS loop over M.n-vectors (x in d_x, overwritten), workspace w laid
// out by lbfgs_layout_n.
static dsm_status run_lbfgs(Minimiser &M, char *w, const size_t off[12], float *d_x, double tol,
                     long long max_iter, dsm_lbfgs_info *info) {
  const int m = M.m;
  M.xb[0] = d_x;
  M.xb[1] = (float *)(w + off[0]);
  M.gb[0] = (float *)(w + off[1]);
  M.gb[1] = (float *)(w + off[2]);
  M.d = (float *)(w + off[3]);
  M.hist = (float *)(w + off[4]);
  M.E[0] = (double *)(w + off[5]);
  M.E[1] = M.E[0] + 1;
  M.dots = (double *)(w + off[6]);
  M.state = (LbState *)(w + off[7]);
  M.vout = (double *)(w + off[7]);  // rb, the state's first member
  M.fe_scr = w + off[8];
  M.vec_scr = w + off[9];
  M.dots_scr = w + off[10];
  const long long n = M.n;
  cudaStream_t st = M.st;
  const int lgrid = (int)std::min<long long>((n + 255) / 256, 152 * 16);
#define CK(expr)                                    \
  do {                                              \
    if ((expr) != cudaSuccess) return DSM_E_CUDA;   \
  } while (0)

  // stored pairs start at zero, so unused slots add nothing to a combination;
  // the fused slope pass's block counter starts at zero
  CK(cudaMemsetAsync(M.hist, 0, (size_t)2 * m * n * sizeof(float), st));
  CK(cudaMemsetAsync(vec_scratch_counter(M.vec_scr), 0, sizeof(unsigned), st));
  lb_init_kernel<<<1, 1, 0, st>>>(M.state);
  CK(cudaGetLastError());
  int cur = 0;  // x = xb[cur], g = gb[cur], E = E[cur]
  CK(M.evaluate(M.xb[0], M.E[0], M.gb[0]));
  CK(vec_dot(n, M.gb[0], M.gb[0], M.vout + 3, nullptr, M.vec_scr, st));
  CK(cudaMemcpyAsync(M.vout + 1, M.E[0], sizeof(double), cudaMemcpyDeviceToDevice, st));
  double rb[6];
  CK(M.read(rb, M.vout, 6));
  double gg = rb[3], f_val = rb[1];
  long long it = 0, evals = 1;
  int converged = 0;
  bool fresh = false;  // gg is that of the current point (read after its last update)
  const double *pending = nullptr;  // the accepted step's dots, not yet folded into the state
  double pending_sy = 0.0;          // and its pair's s.y
  while (it < max_iter) {
    // the pair update and the direction on the device, then the first trial
    // (a = 1), whose read also brings |g|^2 of the current point and the
    // direction's slope
    lb_step_kernel<<<1, 32, 0, st>>>(M.state, pending, m, pending_sy);
    CK(cudaGetLastError());
    pending = nullptr;
    const float *x = M.xb[cur];
    float *xt = M.xb[cur ^ 1];
    const float *g = M.gb[cur];
    float *gt = M.gb[cur ^ 1];
    double *Et = M.E[cur ^ 1];
    lb_lincomb_kernel<<<lgrid, 256, 0, st>>>(n, 2 * m, M.hist, n, M.state, g, M.d);
    CK(cudaGetLastError());
    double a = 1.0;
    CK(M.trial(a, x, xt, Et, gt, rb));
    double df = rb[0], f = rb[1];
    const double dg0 = rb[2];
    gg = rb[3];
    const bool pairs = rb[4] > 0.0;
    const int nxt = (int)rb[5];
    fresh = true;
    if (!isfinite(gg) || !isfinite(f_val)) {
      info->iterations = it;
      info->evaluations = evals;
      info->energy = f_val;
      info->rms_grad = sqrt(gg / n);
      return DSM_E_NONFINITE;
    }
    if (sqrt(gg / n) < tol) {  // converged at x: the trial is not taken
      converged = 1;
      break;
    }

    // strong-Wolfe line search with the approximate-Wolfe test near FP32 noise
    const double c1 = 1e-4, c2 = 0.9, noise = 1e-6 * fabs(f_val);
    const int max_trials = 20;
    auto too_high = [&](double a, double f, double df) {
      if (fabs(f - f_val) <= noise) return df > (2.0 * c1 - 1.0) * dg0;
      return f > f_val + c1 * a * dg0;
    };
    int trials = 1;
    double a_prev = 0.0, f_prev = f_val, d_prev = dg0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    bool bracketed = false, done = false;
    double step = 0.0, last = a;
    while (true) {
      if (too_high(a, f, df) || (trials > 1 && f >= f_prev && fabs(f - f_val) > noise)) {
        lo[0] = a_prev; lo[1] = f_prev; lo[2] = d_prev;
        hi[0] = a; hi[1] = f; hi[2] = df;
        bracketed = true;
        break;
      }
      if (fabs(df) <= -c2 * dg0) {
        step = a;
        done = true;
        break;
      }
      if (df >= 0.0) {
        lo[0] = a; lo[1] = f; lo[2] = df;
        hi[0] = a_prev; hi[1] = f_prev; hi[2] = d_prev;
        bracketed = true;
        break;
      }
      a_prev = a;
      f_prev = f;
      d_prev = df;
      if (trials >= max_trials) break;
      a *= 2.0;
      CK(M.trial(a, x, xt, Et, gt, rb));
      df = rb[0];
      f = rb[1];
      trials++;
      last = a;
    }
    if (!done && !bracketed) step = a_prev;  // never bracketed: the last descending point
    while (!done && bracketed && trials < max_trials) {
      a = cubic_step(lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]);
      CK(M.trial(a, x, xt, Et, gt, rb));
      df = rb[0];
      f = rb[1];
      trials++;
      last = a;
      if (too_high(a, f, df) || (f >= lo[1] && fabs(f - f_val) > noise)) {
        hi[0] = a; hi[1] = f; hi[2] = df;
      } else {
        if (fabs(df) <= -c2 * dg0) {
          step = a;
          done = true;
          break;
        }
        if (df * (hi[0] - lo[0]) >= 0.0) {
          hi[0] = lo[0]; hi[1] = lo[1]; hi[2] = lo[2];
        }
        lo[0] = a; lo[1] = f; lo[2] = df;
      }
    }
    if (!done && bracketed) step = lo[0];
    evals += trials;
    if (!(step > 0.0)) {
      if (pairs) {  // drop the pairs and retry by steepest descent
        lb_reset_kernel<<<1, 1, 0, st>>>(M.state);
        CK(cudaGetLastError());
        continue;
      }
      break;
    }
    if (last != step) {  // the accepted point is not the last one evaluated
      CK(M.trial(step, x, xt, Et, gt, rb));
      df = rb[0];
      f = rb[1];
      evals++;
    }
    // new pair s = step d, y = g_new - g into slot nxt; every stored s, y
    // against g_new in one batched pass (the new pair's included), then y.y,
    // g_new.g_new and s.s; s.y = step (g_new.d - g.d) from the slopes.  The
    // device folds them into its state (no host read).
    float *s_new = M.hist + (size_t)nxt * n;
    float *y_new = M.hist + (size_t)(m + nxt) * n;
    const double minus1 = -1.0;
    CK(vec_axpby(n, step, M.d, 0.0, s_new, st));
    CK(vec_lincomb(n, 1, g, n, &minus1, gt, 1.0, y_new, st));
    CK(vec_dots(n, 2 * m, M.hist, n, gt, M.dots, M.dots_scr, st));
    CK(vec_sumsq3(n, y_new, gt, s_new, M.dots + 2 * m, M.dots_scr, st));
    pending = M.dots;  // folded in by the next iteration's lb_step_kernel
    pending_sy = step * (df - dg0);
    fresh = false;
    cur ^= 1;
    f_val = f;
    it++;
  }
#undef CK
  // the minimiser's current point back into the caller's buffer
  if (cur != 0 &&
      cudaMemcpyAsync(d_x, M.xb[cur], n * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return DSM_E_CUDA;
  if (!fresh) {  // |g|^2 of the last accepted point (its dots hold g.g)
    if (M.read(rb, M.dots + 2 * m + 1, 1) != cudaSuccess) return DSM_E_CUDA;
    gg = rb[0];
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return DSM_E_CUDA;
  info->iterations = it;
  info->evaluations = evals;
  info->energy = f_val;
  info->rms_grad = sqrt(gg / n);
  info->converged = converged;
  return DSM_OK;
}

extern "C" {

dsm_status dsm_lbfgs_compact(int k, const double *SY, const double *YY, const double *a,
                             const double *b, double gamma, double *cx, double *cs, double *cy) {
  if (k < 1 || !SY || !YY || !a || !b || !cx || !cs || !cy) return DSM_E_INVAL;
  std::vector<int> ord(k);
  for (int i = 0; i < k; i++) ord[i] = i;
  std::vector<double> w(k), z(k), u(k);
  return compact_slots(k, ord.data(), k, SY, YY, a, b, gamma, w.data(), z.data(), u.data(), cx,
                       cs, cy)
             ? DSM_OK
             : DSM_E_INVAL;
}

// Workspace of an L-BFGS run over n-vectors whose energy needs fe_bytes of
// scratch.
static size_t lbfgs_layout_n(long long n, int m, size_t fe_bytes, size_t off[12]) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += (size_t)round_up((long long)bytes, 256);
    return at;
  };
  off[0] = take(n * sizeof(float));               // second x buffer
  off[1] = take(n * sizeof(float));               // g
  off[2] = take(n * sizeof(float));               // gt
  off[3] = take(n * sizeof(float));               // d
  off[4] = take((size_t)2 * m * n * sizeof(float));  // s_0..s_{m-1}, y_0..y_{m-1}
  off[5] = take(2 * sizeof(double));              // E, Et
  off[6] = take((size_t)(2 * m + 3) * sizeof(double));  // S^T g, Y^T g, then y.y, g.g, s.s
  off[7] = take(sizeof(LbState));                 // the pair bookkeeping on the device
  off[8] = take(fe_bytes);
  off[9] = take(vec_scratch_bytes(n));
  off[10] = take(vec_dots_scratch_bytes(n, 4 * m));
  return o;
}

static size_t lbfgs_layout(const dsm_params *p, int m, size_t off[12]) {
  return lbfgs_layout_n((long long)p->nx * p->ny * p->nz, m,
                        fe_scratch_bytes(p->lattice, p->nx, p->ny, p->nz), off);
}

dsm_status dsm_lbfgs_workspace_bytes(const dsm_params *p, int m, size_t *bytes) {
  if (!p || !bytes || m < 1 || 2 * m > LINCOMB_MAX) return DSM_E_INVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return DSM_E_INVAL;
  size_t off[12];
  *bytes = lbfgs_layout(p, m, off);
  return DSM_OK;
}

dsm_status dsm_lbfgs_minimize(const dsm_params *p, const float *d_fixed,
                              const unsigned char *d_mask, int active, double dP, double kcs,
                              double V0, double fg, float *d_x, int m, double tol,
                              long long max_iter, void *d_work, size_t work_bytes,
                              dsm_lbfgs_info *info, void *cuda_stream) {
  TraceRange trace_range("L-BFGS");
  if (!p || !d_fixed || !d_x || !d_work || !info) return DSM_E_INVAL;
  if (active != 1 && active != 2) return DSM_E_INVAL;
  if (active == 1 && !d_mask) return DSM_E_INVAL;
  if (p->lattice != DSM_D2Q9 && p->lattice != DSM_D3Q19) return DSM_E_INVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->lattice == DSM_D2Q9 && p->nz != 1))
    return DSM_E_INVAL;
  if ((long long)p->nx * p->ny * p->nz >= (1ll << 31)) return DSM_E_INVAL;
  if (m < 1 || 2 * m > LINCOMB_MAX || max_iter < 0 || !(tol >= 0.0) || kcs < 0.0)
    return DSM_E_INVAL;
  double kap[3];
  dsm_status s = dsm_kappa(p, kap);
  if (s != DSM_OK) return s;
  size_t off[12];
  if (work_bytes < lbfgs_layout(p, m, off) || ((uintptr_t)d_work & 255u)) return DSM_E_WORKSPACE;
  memset(info, 0, sizeof(*info));

  Minimiser M;
  M.n = (long long)p->nx * p->ny * p->nz;
  M.m = m;
  M.st = (cudaStream_t)cuda_stream;
  s = fe_args_of(p, kap, active, fg, &M.fa);
  if (s != DSM_OK) return s;
  M.fa.mask = d_mask;
  M.kind = p->lattice;
  M.dP = dP;
  M.kcs = kcs;
  M.V0 = V0;
  M.fixed = d_fixed;
  M.active = active;
  return run_lbfgs(M, (char *)d_work, off, d_x, tol, max_iter, info);
}

dsm_status dsm_lbfgs_multi_workspace_bytes(const dsm_params *p, int nfluid, int m,
                                           size_t *bytes) {
  if (!p || !bytes || m < 1 || 2 * m > LINCOMB_MAX) return DSM_E_INVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return DSM_E_INVAL;
  if (p->lattice != DSM_D2Q9 && p->lattice != DSM_D3Q19) return DSM_E_INVAL;
  if (nfluid < 2 || nfluid > FEM_MAX_NF + 1) return DSM_E_INVAL;
  size_t off[12];
  const long long nodes = (long long)p->nx * p->ny * p->nz;
  *bytes = lbfgs_layout_n(nodes * (nfluid - 1), m,
                          fe_multi_scratch_bytes(p->lattice, p->nx, p->ny, p->nz, nfluid - 1),
                          off);
  return DSM_OK;
}

dsm_status dsm_lbfgs_minimize_multi(const dsm_params *p, int nfluid, const double *kappa,
                                    const float *d_c1, const double *dP, const double *kcs,
                                    const double *V0, float *d_x, int m, double tol,
                                    long long max_iter, void *d_work, size_t work_bytes,
                                    dsm_lbfgs_info *info, void *cuda_stream) {
  TraceRange trace_range("N-fluid L-BFGS");
  if (!d_c1 || !d_x || !d_work || !info) return DSM_E_INVAL;
  if (m < 1 || 2 * m > LINCOMB_MAX || max_iter < 0 || !(tol >= 0.0)) return DSM_E_INVAL;
  Minimiser M;
  dsm_status s = fem_args_of(p, nfluid, kappa, dP, kcs, V0, &M.fm, &M.fcons);
  if (s != DSM_OK) return s;
  const long long nodes = (long long)p->nx * p->ny * p->nz;
  size_t off[12];
  const size_t need = lbfgs_layout_n(
      nodes * (nfluid - 1), m, fe_multi_scratch_bytes(p->lattice, p->nx, p->ny, p->nz, nfluid - 1),
      off);
  if (work_bytes < need || ((uintptr_t)d_work & 255u)) return DSM_E_WORKSPACE;
  memset(info, 0, sizeof(*info));
  M.multi = true;
  M.fm.c1 = d_c1;
  M.n = nodes * (nfluid - 1);
  M.m = m;
  M.st = (cudaStream_t)cuda_stream;
  M.kind = p->lattice;
  M.fixed = d_c1;
  M.active = 2;
  return run_lbfgs(M, (char *)d_work, off, d_x, tol, max_iter, info);
}

}  // extern "C"
