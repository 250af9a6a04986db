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
// and one linear combination per iteration.  Device work per iteration: about
// a dozen launches and two host reads.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dsm_em.cuh"
#include "dsm_trace.cuh"

using namespace dsm;

namespace {

// Compact-form coefficients: R w = a, R^T u = (D + gamma YY) w - gamma b,
// d = -gamma g - S u + gamma Y w.  SY, YY: k x k row-major (pairs oldest
// first), R the upper triangle of SY, D its diagonal.
bool compact(int k, const double *SY, const double *YY, const double *a, const double *b,
             double gamma, double *cx, double *cs, double *cy) {
  std::vector<double> w(k), z(k), u(k);
  for (int i = k - 1; i >= 0; i--) {  // back substitution, R upper triangular
    double v = a[i];
    for (int j = i + 1; j < k; j++) v -= SY[i * k + j] * w[j];
    if (!(SY[i * k + i] != 0.0)) return false;
    w[i] = v / SY[i * k + i];
  }
  for (int i = 0; i < k; i++) {
    double v = SY[i * k + i] * w[i] - gamma * b[i];
    for (int j = 0; j < k; j++) v += gamma * YY[i * k + j] * w[j];
    z[i] = v;
  }
  for (int i = 0; i < k; i++) {  // forward substitution, R^T lower triangular
    double v = z[i];
    for (int j = 0; j < i; j++) v -= SY[j * k + i] * u[j];
    u[i] = v / SY[i * k + i];
  }
  *cx = -gamma;
  for (int i = 0; i < k; i++) {
    cs[i] = -u[i];
    cy[i] = gamma * w[i];
  }
  return true;
}

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
  double *E[2], *dots, *vout;
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
  // trial point xt = x + a d: energy and directional derivative
  cudaError_t trial(double a, const float *x, float *xt, double *Et, float *gt, double *f,
                    double *df) {
    cudaError_t e = vec_lincomb(n, 1, d, n, &a, x, 1.0, xt, st);
    if (e == cudaSuccess) e = evaluate(xt, Et, gt);
    if (e == cudaSuccess) e = vec_dot(n, gt, d, vout, nullptr, vec_scr, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vout + 1, Et, sizeof(double), cudaMemcpyDeviceToDevice, st);
    double h[2];
    if (e == cudaSuccess) e = read(h, vout, 2);
    *df = h[0];
    *f = h[1];
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
  M.vout = (double *)(w + off[7]);
  M.fe_scr = w + off[8];
  M.vec_scr = w + off[9];
  M.dots_scr = w + off[10];
  const long long n = M.n;
  cudaStream_t st = M.st;
#define CK(expr)                                    \
  do {                                              \
    if ((expr) != cudaSuccess) return DSM_E_CUDA;   \
  } while (0)

  // stored pairs start at zero, so unused slots add nothing to a combination
  CK(cudaMemsetAsync(M.hist, 0, (size_t)2 * m * n * sizeof(float), st));
  int cur = 0;  // x = xb[cur], g = gb[cur], E = E[cur]
  CK(M.evaluate(M.xb[0], M.E[0], M.gb[0]));
  CK(vec_dot(n, M.gb[0], M.gb[0], M.vout, nullptr, M.vec_scr, st));
  CK(cudaMemcpyAsync(M.vout + 1, M.E[0], sizeof(double), cudaMemcpyDeviceToDevice, st));
  double h2[2];
  CK(M.read(h2, M.vout, 2));
  double gg = h2[0], f_val = h2[1];
  std::vector<int> order;  // slots of the stored pairs, oldest first
  int nxt = 0;
  double gamma = 1.0;
  std::vector<double> SY((size_t)m * m, 0.0), YY((size_t)m * m, 0.0), Ag(m, 0.0), Bg(m, 0.0);
  std::vector<double> coef(2 * m, 0.0), hv(4 * m + 2, 0.0);
  long long it = 0, evals = 1;
  int converged = 0;
  while (it < max_iter) {
    if (!isfinite(gg) || !isfinite(f_val)) {
      info->iterations = it;
      info->evaluations = evals;
      info->energy = f_val;
      info->rms_grad = sqrt(gg / n);
      return DSM_E_NONFINITE;
    }
    if (sqrt(gg / n) < tol) {
      converged = 1;
      break;
    }
    const int k = (int)order.size();
    double cx = 0.0, dg0 = 0.0;
    bool ok = false;
    std::fill(coef.begin(), coef.end(), 0.0);
    if (k > 0) {
      std::vector<double> sy(k * k), yy(k * k), a(k), b(k), cs(k), cy(k);
      for (int i = 0; i < k; i++) {
        a[i] = Ag[order[i]];
        b[i] = Bg[order[i]];
        for (int j = 0; j < k; j++) {
          sy[i * k + j] = SY[(size_t)order[i] * m + order[j]];
          yy[i * k + j] = YY[(size_t)order[i] * m + order[j]];
        }
      }
      if (compact(k, sy.data(), yy.data(), a.data(), b.data(), gamma, &cx, cs.data(), cy.data())) {
        dg0 = cx * gg;
        for (int i = 0; i < k; i++) {
          coef[order[i]] = cs[i];
          coef[m + order[i]] = cy[i];
          dg0 += cs[i] * a[i] + cy[i] * b[i];
        }
        ok = dg0 < 0.0;
      }
    }
    if (!ok) {  // no pairs, or not a descent direction: steepest descent
      order.clear();
      std::fill(coef.begin(), coef.end(), 0.0);
      cx = -1.0 / std::max(sqrt(gg), 1e-300);
      dg0 = cx * gg;
    }
    const float *x = M.xb[cur];
    float *xt = M.xb[cur ^ 1];
    const float *g = M.gb[cur];
    float *gt = M.gb[cur ^ 1];
    double *Et = M.E[cur ^ 1];
    CK(vec_lincomb(n, order.empty() ? 0 : 2 * m, M.hist, n, coef.data(), g, cx, M.d, st));

    // strong-Wolfe line search with the approximate-Wolfe test near FP32 noise
    const double c1 = 1e-4, c2 = 0.9, noise = 1e-6 * fabs(f_val);
    const int max_trials = 20;
    auto too_high = [&](double a, double f, double df) {
      if (fabs(f - f_val) <= noise) return df > (2.0 * c1 - 1.0) * dg0;
      return f > f_val + c1 * a * dg0;
    };
    int trials = 0;
    double a_prev = 0.0, f_prev = f_val, d_prev = dg0, a = 1.0, f = 0.0, df = 0.0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    bool bracketed = false, done = false;
    double step = 0.0, last = -1.0;
    while (trials < max_trials) {
      CK(M.trial(a, x, xt, Et, gt, &f, &df));
      trials++;
      last = a;
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
      a *= 2.0;
    }
    if (!done && !bracketed) step = a_prev;  // never bracketed: the last descending point
    while (!done && bracketed && trials < max_trials) {
      a = cubic_step(lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]);
      CK(M.trial(a, x, xt, Et, gt, &f, &df));
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
      if (!order.empty()) {
        order.clear();
        continue;
      }
      break;
    }
    if (last != step) {  // the accepted point is not the last one evaluated
      CK(M.trial(step, x, xt, Et, gt, &f, &df));
      evals++;
    }
    // new pair s = step d, y = g_new - g into slot nxt (the oldest pair leaves a full ring)
    order.erase(std::remove(order.begin(), order.end(), nxt), order.end());
    float *s_new = M.hist + (size_t)nxt * n;
    float *y_new = M.hist + (size_t)(m + nxt) * n;
    const double minus1 = -1.0;
    CK(vec_axpby(n, step, M.d, 0.0, s_new, st));
    CK(vec_lincomb(n, 1, g, n, &minus1, gt, 1.0, y_new, st));
    // every stored s, y against y_new and against g_new, in one batched pass
    CK(vec_dots2(n, 2 * m, M.hist, n, y_new, gt, M.dots, M.dots_scr, st));
    CK(vec_dot(n, s_new, s_new, M.dots + 4 * m, nullptr, M.vec_scr, st));
    CK(vec_dot(n, gt, gt, M.dots + 4 * m + 1, nullptr, M.vec_scr, st));
    CK(M.read(hv.data(), M.dots, 4 * m + 2));  // the iteration's one read after the step
    const double ss = hv[4 * m], sy = hv[nxt], yy = hv[m + nxt];
    gg = hv[4 * m + 1];
    for (int i = 0; i < m; i++) {
      Ag[i] = hv[2 * m + i];
      Bg[i] = hv[3 * m + i];
    }
    if (sy > 1e-12 * sqrt(ss * yy)) {
      for (int i = 0; i < m; i++) {
        SY[(size_t)i * m + nxt] = hv[i];     // s_i . y_new
        YY[(size_t)i * m + nxt] = hv[m + i];  // y_i . y_new
        YY[(size_t)nxt * m + i] = hv[m + i];
      }
      gamma = sy / yy;
      order.push_back(nxt);
      nxt = (nxt + 1) % m;
    }
    cur ^= 1;
    f_val = f;
    it++;
  }
#undef CK
  // the minimiser's current point back into the caller's buffer
  if (cur != 0 &&
      cudaMemcpyAsync(d_x, M.xb[cur], n * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return DSM_E_CUDA;
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
  return compact(k, SY, YY, a, b, gamma, cx, cs, cy) ? DSM_OK : DSM_E_INVAL;
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
  off[6] = take((size_t)(4 * m + 2) * sizeof(double));  // batched dots, then s.s and g.g
  off[7] = take(4 * sizeof(double));              // single dots
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
