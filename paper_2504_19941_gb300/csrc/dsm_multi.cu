// dsm_multi.cu -- the lattice Boltzmann step for N fluid components on a frozen
// diffuse solid (Sec. II.B states the method for the N + 1-component model and
// demonstrates N = 2; here N = 2 .. 4).  Population form, FP64 or FP32
// storage and arithmetic; every free fluid C_2 .. C_N has its own
// Cahn-Hilliard populations g_f, and C_{N+1} = 1 - C_1 - sum_f C_f.
//
// Per step, as for two fluids: a moments pass (C_f = sum_i g_f,i after the
// pull) and a fused pass (pull f and g with interpolated bounce-back and the
// face rules; chemical potentials, density and relaxation maps, forces,
// moments; BGK collision of f and of every g_f).  Readings for N > 2, each
// reducing to the two-fluid one:
//   mu_f = d_f - d_{N+1},  d_k = kappa_k b(C_k) - alpha^2 kappa_k L[C_k]
//     (the exact derivative of the N-fluid free energy);
//   F = sum_f mu_f G[C_f] + C_2 b (the potential form for every fluid, the
//     body force on fluid 2);
//   rho = rho_{N+1} + sum_f (rho_f - rho_{N+1}) phi_f, phi_f = C_f / (1 - C_1)
//     clamped to [0, 1] (0 where 1 - C_1 <= 1e-6);
//   tau = the relaxation time of the locally largest fluid concentration,
//     ties to the later fluid.
// At tau_g = 1 with periodic faces every g_f is held as g_eq, as for two
// fluids: the post-collision g_f is g_eq fixed by (A_f = mu_f - 3/2 C_f u.u,
// C_f, u), so the fused pass stores A_f and the shared u instead of Q
// populations per fluid, and the moments pass rebuilds each C_f from its
// neighbours' (A_f, C_f, u) with the two-fluid form's arithmetic.
#include <math.h>
#include <string.h>

#include <new>

#include "dsm_lb_impl.cuh"
#include "dsm_pair.cuh"
#include "dsm_tmap.cuh"
#include "dsm_trace.cuh"

namespace dsm {

constexpr int ML_MAX_NF = 3;  // free fluids (N - 1)

template <class T>
struct MLArgs {
  int nx, ny, nz;
  long long N, pitch;
  int face[6];
  int walls;
  T kappa[ML_MAX_NF + 2];            // kappa_1, the free fluids', the dependent fluid's
  T rho[ML_MAX_NF + 1], om[ML_MAX_NF + 1];  // per fluid: density, 1 / tau
  T omg, a2, alpha_s;
  T irho;                // 1 / rho of the dependent fluid (every rho when they are equal)
  T body[3];
  int rc;                // the fluids' densities differ (else rho is constant)
  const T *f_in, *g_in;  // Q planes; NF x Q planes (fluid-major)
  T *f_out, *g_out;
  // the f planes one by one (fin[j] = f_in + j pitch): a pull or a store
  // addresses its plane from a kernel parameter, with no 64-bit multiply
  const T *fin[19];
  T *fout[19];
  T *C;                  // NF planes: the moments pass output
  const T *Cprev;        // g_eq form: NF planes, C of the state's last collision
  T *A;                  // g_eq form: NF planes of A_f = mu_f - 3/2 C_f u.u
  T *U;                  // g_eq form: u_x, u_y, u_z planes
  const T *C1;
  T *out;                // fields mode: one plane
  int field, index;
  int *err;              // latched error word (bits ERR_NONFINITE, ERR_TIMEOUT, ERR_BOUNDS)
  // single-pass step (dsm_mlz.cuh): the padded output buffers, their widths
  T *Qz, *Uz, *Pz;
  int nxp, nyp;
};

template <class T>
__device__ __forceinline__ const T *plane(const T *base, long long pitch, int k) {
  return base + (long long)k * pitch;
}
template <class T>
__device__ __forceinline__ T *plane(T *base, long long pitch, int k) {
  return base + (long long)k * pitch;
}

// moments pass: C_f(x) = sum_i g_f,i pulled into x (face rules on the faces;
// FC: the lattice has a mirror or wall face, else the face code is compiled out)
template <int K, class T, int NF, bool FC>
__global__ void __launch_bounds__(256) ml_moments_kernel(MLArgs<T> a) {
  using L = Lat<K>;
  constexpr int Q = L::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x >= a.nx || y >= a.ny || z >= a.nz) return;
  Hood h;
  if constexpr (FC) h.init_faces(x, y, z, a.nx, a.ny, a.nz, a.face);
  else h.init(x, y, z, a.nx, a.ny, a.nz);
  h.guard(a.err);
  const int n = h.g(h.ox[1] + h.oy[1] + h.oz[1]);
  const bool edge = FC && on_wall_face(a.face, x, y, z, a.nx, a.ny, a.nz);
#pragma unroll
  for (int f = 0; f < NF; f++) {
    const T *g = a.g_in + (long long)f * Q * a.pitch;
    T s = T(0);
    if (edge) {
#pragma unroll
      for (int i = 1; i < Q; i++) {
        int k = i, src = h.plus_rt<L>(L::opp(i));
        if (face_cross<L>(a.face, x, y, z, a.nx, a.ny, a.nz, i, &k) == 2) src = n;
        s += plane(g, a.pitch, k)[src];
      }
    } else {
#pragma unroll
      for (int i = 1; i < Q; i++) s += __ldg(plane(g, a.pitch, i) + h.minus<L>(i));
    }
    a.C[f * a.pitch + n] = plane(g, a.pitch, 0)[n] + s;
  }
}

// moments pass with g held as g_eq: C_f(x) = sum_i g_eq_i(x - c_i) from the
// neighbours' (A_f, C_f, u), through the two-fluid form's per-node arithmetic
template <int K, class T, int NF>
__global__ void __launch_bounds__(256) ml_moments_eq_kernel(MLArgs<T> a) {
  using L = Lat<K>;
  constexpr int Q = L::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x >= a.nx || y >= a.ny || z >= a.nz) return;
  Hood h;
  h.init(x, y, z, a.nx, a.ny, a.nz);
  h.guard(a.err);
  const int n = h.g(h.ox[1] + h.oy[1] + h.oz[1]);
  T uy[Q][3];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const int m = i == 0 ? n : h.minus<L>(i);
    uy[i][0] = (i == 0 || L::cx(i)) ? __ldg(a.U + m) : T(0);
    uy[i][1] = (i == 0 || L::cy(i)) ? __ldg(a.U + a.pitch + m) : T(0);
    uy[i][2] = (L::D == 3 && (i == 0 || L::cz(i))) ? __ldg(a.U + 2 * a.pitch + m) : T(0);
  }
#pragma unroll
  for (int f = 0; f < NF; f++) {
    T Ay[Q], Cy[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const int m = i == 0 ? n : h.minus<L>(i);
      Ay[i] = __ldg(a.A + f * a.pitch + m);
      Cy[i] = __ldg(a.Cprev + f * a.pitch + m);
    }
    a.C[f * a.pitch + n] = moments_eq_node<L, T>(Ay, Cy, uy);
  }
}

// rho of the volume fractions at one point.  One reciprocal of 1 - C1 per
// point; in FP32 the fast reciprocal (within 2 ulp) serves, since every
// fraction is clamped to [0, 1] right after.
template <class T, int NF>
__device__ __forceinline__ T ml_rho(const MLArgs<T> &a, const T (&c)[NF], T c1) {
  const T den = T(1) - c1;
  T r = a.rho[NF];
  if (!(den > T(1e-6))) return r;
  T inv;
  if constexpr (sizeof(T) == 4) inv = __fdividef(1.0f, den);
  else inv = T(1) / den;
#pragma unroll
  for (int f = 0; f < NF; f++) {
    T ph = c[f] * inv;
    ph = ph < T(0) ? T(0) : (ph > T(1) ? T(1) : ph);
    r += (a.rho[f] - a.rho[NF]) * ph;
  }
  return r;
}

enum { ML_STEP = 0, ML_FIELDS = 1 };

// The fused pass's view of the neighbourhood in the two-pass step: C1 and the
// free fluids' C from their global planes (the moments pass wrote this step's
// C), the g_eq state (A_f, u) to its canonical planes.  The single-pass step
// (dsm_mlz.cuh) reads C1 and C from shared memory instead.
template <class T>
struct MLGlobalIO {
  static constexpr bool kSolidFirst = false;  // pull f at every node
  static constexpr bool kZ = false;           // canonical layout, faces at run time
  static constexpr bool kUnrollWall = false;  // wall links in a rolled loop
  template <class L>
  __device__ __forceinline__ T C1(const MLArgs<T> &a, const Hood &h, int n, int i) const {
    return i == 0 ? a.C1[n] : __ldg(a.C1 + h.plus<L>(i));
  }
  template <class L>
  __device__ __forceinline__ T C(const MLArgs<T> &a, const Hood &h, int n, int f, int i) const {
    return i == 0 ? a.C[f * a.pitch + n] : __ldg(a.C + f * a.pitch + h.plus<L>(i));
  }
  template <class L, int NF>
  __device__ __forceinline__ void put_eq(const MLArgs<T> &a, long long n, const T (&A)[NF],
                                         const T (&)[NF], const T (&u)[3]) const {
#pragma unroll
    for (int f = 0; f < NF; f++) a.A[f * a.pitch + n] = A[f];
    a.U[n] = u[0];
    a.U[a.pitch + n] = u[1];
    if (L::D == 3) a.U[2 * a.pitch + n] = u[2];
  }
};

// FC: the lattice has a mirror or wall face (populations only); without one the
// face code is compiled out, which keeps the periodic step's register count
// RCV: the fluids' densities may differ (a.rc decides at run time); false:
// they are equal (a.rc = 0), and the density map, its gradient and the terms
// they enter are compiled out -- rho is the common density, G[rho] = 0, the
// same results bit for bit.
template <int K, class T, int NF, int MODE, bool EQ, bool FC, class IO = MLGlobalIO<T>,
          bool RCV = true>
__device__ __forceinline__ void ml_node_body(const MLArgs<T> &a, int x, int y, int z,
                                             const IO &io = IO()) {
  static_assert(!(EQ && FC), "the g_eq form is periodic only");
  using L = Lat<K>;
  constexpr int Q = L::Q;
  constexpr int NC = NF + 2;
  if (x >= a.nx || y >= a.ny || z >= a.nz) return;
  Hood h;
  // RTF: face offsets and the interpolated bounce-back's face check at run
  // time.  The two-pass g_eq variant keeps them although its faces are
  // periodic: with them compiled out its schedule changed and the step took
  // 13 % longer.
  constexpr bool RTF = FC || (EQ && !IO::kZ);
  if constexpr (RTF) h.init_faces(x, y, z, a.nx, a.ny, a.nz, a.face);
  else h.init(x, y, z, a.nx, a.ny, a.nz);
  h.guard(a.err);
  const int n = h.g(h.ox[1] + h.oy[1] + h.oz[1]);

  // ---- the neighbourhood: C1 and the free fluids, stencils of every component
  T cv[NC], lap[NC], gC[NF][3], gR[3] = {T(0), T(0), T(0)}, gc1[3] = {T(0), T(0), T(0)};
  unsigned nb_solid = 0;  // bit i: x + c_i is solid
  T c1max = T(0);         // one-pass form: the largest C1 of the neighbours
  cv[0] = io.template C1<L>(a, h, n, 0);
  T last = T(1) - cv[0];
#pragma unroll
  for (int f = 0; f < NF; f++) {
    cv[1 + f] = io.template C<L>(a, h, n, f, 0);
    last -= cv[1 + f];
  }
  cv[NC - 1] = last;
#pragma unroll
  for (int k = 0; k < NC; k++) lap[k] = T(0);
#pragma unroll
  for (int f = 0; f < NF; f++) gC[f][0] = gC[f][1] = gC[f][2] = T(0);
  // (gradient components only where c_i has one: w 0 c is an operation IEEE
  // arithmetic cannot drop, and for finite values it adds nothing.)  The
  // Laplacian sums of C1 and the free fluids go in pairs of components, the
  // gradient of two free fluids as one pair per component (dsm_pair.cuh).
  constexpr int NP = (NF + 1) / 2;  // pairs among components 0 .. NF
  Pr<T> lapP[NP > 0 ? NP : 1], mctr[NP > 0 ? NP : 1];
#pragma unroll
  for (int k = 0; k < NP; k++) {
    lapP[k] = pr(T(0), T(0));
    mctr[k] = pr(-cv[2 * k], -cv[2 * k + 1]);
  }
#pragma unroll
  for (int i = 1; i < Q; i++) {
    const T w = T(L::w(i));
    const T cx = T(L::cx(i)), cy = T(L::cy(i)), cz = T(L::cz(i));
    const T c1m = io.template C1<L>(a, h, n, i);
    T cm[NF], val[NF + 1];
    val[0] = c1m;
#pragma unroll
    for (int f = 0; f < NF; f++) {
      cm[f] = io.template C<L>(a, h, n, f, i);
      val[1 + f] = cm[f];
    }
#pragma unroll
    for (int k = 0; k < NP; k++)
      lapP[k] = pr_fma(pr(w, w), pr_add(pr(val[2 * k], val[2 * k + 1]), mctr[k]), lapP[k]);
    if constexpr ((NF + 1) % 2) lap[NF] += w * (val[NF] - cv[NF]);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const int cd = d == 0 ? L::cx(i) : (d == 1 ? L::cy(i) : L::cz(i));
      if (cd) {
        const T wc = w * T(cd);
#pragma unroll
        for (int f = 0; f + 1 < NF; f += 2) {
          const Pr<T> gg = pr_fma(pr(wc, wc), pr(cm[f], cm[f + 1]), pr(gC[f][d], gC[f + 1][d]));
          gC[f][d] = gg.a;
          gC[f + 1][d] = gg.b;
        }
        if constexpr (NF % 2) gC[NF - 1][d] += wc * cm[NF - 1];
      }
    }
    if (RCV && a.rc) {
      const T r = w * ml_rho<T, NF>(a, cm, c1m);
      if (L::cx(i)) gR[0] += r * cx;
      if (L::cy(i)) gR[1] += r * cy;
      if (L::cz(i)) gR[2] += r * cz;
    }
    if constexpr (IO::kZ) {
      c1max = c1max > c1m ? c1max : c1m;
    } else {
      if (L::cx(i)) gc1[0] += w * cx * c1m;
      if (L::cy(i)) gc1[1] += w * cy * c1m;
      if (L::cz(i)) gc1[2] += w * cz * c1m;
      if (c1m >= T(0.5)) nb_solid |= 1u << i;
    }
  }
  // one-pass form: the wall-link bits and G[C1] only at a fluid node with a
  // solid neighbour, from C1 in shared memory again (the same sums, in the
  // same order); elsewhere one running maximum of C1 settles it
  if constexpr (IO::kZ) {
    if (c1max >= T(0.5) && !(cv[0] >= T(0.5))) {
#pragma unroll
      for (int i = 1; i < Q; i++) {
        const T w = T(L::w(i));
        const T c1m = io.template C1<L>(a, h, n, i);
        if (L::cx(i)) gc1[0] += w * T(L::cx(i)) * c1m;
        if (L::cy(i)) gc1[1] += w * T(L::cy(i)) * c1m;
        if (L::cz(i)) gc1[2] += w * T(L::cz(i)) * c1m;
        if (c1m >= T(0.5)) nb_solid |= 1u << i;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NP; k++) {
    lap[2 * k] = lapP[k].a;
    lap[2 * k + 1] = lapP[k].b;
  }
  // the dependent fluid C_{N+1} = 1 - C_1 - sum_f C_f: its Laplacian by the
  // stencil's linearity, L[C_{N+1}] = -L[C_1] - sum_f L[C_f] (sum_i w_i (1 - 1) = 0)
  lap[NC - 1] = -lap[0];
#pragma unroll
  for (int f = 0; f < NF; f++) lap[NC - 1] -= lap[1 + f];
  T mu[NF], F[3] = {T(0), T(0), T(0)};
  T d[NC];
#pragma unroll
  for (int k = 0; k < NC; k++)
    d[k] = a.kappa[k] * bwell(cv[k]) - a.a2 * a.kappa[k] * (T(6) * lap[k]);
#pragma unroll
  for (int f = 0; f < NF; f++) {
    mu[f] = d[1 + f] - d[NC - 1];
    for (int e = 0; e < 3; e++) F[e] += mu[f] * (T(3) * gC[f][e]);
  }
  for (int e = 0; e < 3; e++) {
    F[e] += cv[1] * a.body[e];
    gR[e] *= T(3);
    gc1[e] *= T(3);
  }
  T cfree[NF];
#pragma unroll
  for (int f = 0; f < NF; f++) cfree[f] = cv[1 + f];
  const T rho = RCV ? ml_rho<T, NF>(a, cfree, cv[0]) : a.rho[NF];
  // relaxation of the locally largest fluid, ties to the later one
  int big = NF;
  T bigc = cv[NC - 1];
#pragma unroll
  for (int f = NF - 1; f >= 0; f--)
    if (cv[1 + f] > bigc) {
      bigc = cv[1 + f];
      big = f;
    }
  const T om = a.om[big];
  const bool solid_x = cv[0] >= T(0.5);

  // ---- pull f and every g_f from x - c_j, all loads issued up front; the
  // rare links (a solid upstream node, a domain face) are corrected below
  // (IO::kSolidFirst: a solid node, whose f is reset to w, pulls nothing)
  T fs[Q], gs[EQ ? 1 : NF][Q];
  const bool pull = !IO::kSolidFirst || !solid_x;
#pragma unroll
  for (int j = 0; j < Q; j++) {
    const int src = h.minus<L>(j);
    fs[j] = pull ? __ldg(a.fin[j] + src) : T(L::w(j));
    if constexpr (!EQ) {
#pragma unroll
      for (int f = 0; f < NF; f++)
        gs[f][j] = __ldg(plane(a.g_in + (long long)f * Q * a.pitch, a.pitch, j) + src);
    }
  }
  // interpolated bounce-back where the upstream node (or its image across a
  // mirror) is solid
  if (!solid_x && (nb_solid & ~1u)) {
    const T cc = cv[0] < T(1e-9) ? T(1e-9) : (cv[0] > T(0.5) ? T(0.5) : cv[0]);
    const T xs = T(2) * a.alpha_s * atanh(T(2) * cc - T(1));
    const T gn = sqrt(gc1[0] * gc1[0] + gc1[1] * gc1[1] + gc1[2] * gc1[2]);
    // IO::kUnrollWall: unrolled over the directions (a warp executes the body
    // of a direction only when one of its nodes has that wall link, and each
    // result lands in a fixed register); else a rolled loop whose result goes
    // through a select over all directions (in the two-pass fused pass the
    // unrolled form ran slower)
    auto link = [&](int j, int i, T q) {
      const T fi_x = a.fin[i][n];
      int ki = i;
      bool second = !((nb_solid >> j) & 1u);
      if (RTF && a.walls && face_cross<L>(a.face, x, y, z, a.nx, a.ny, a.nz, i, &ki) == 2)
        second = false;
      if (q < T(0.5) && second)
        return T(2) * q * fi_x + (T(1) - T(2) * q) * a.fin[ki][h.plus_rt<L>(j)];
      if (q < T(0.5)) return fi_x;
      return (T(1) / (T(2) * q)) * fi_x + (T(1) - T(1) / (T(2) * q)) * a.fin[j][n];
    };
    if constexpr (IO::kUnrollWall) {
#pragma unroll
      for (int j = 1; j < Q; j++) {
        const int i = L::opp(j);
        if ((nb_solid >> i) & 1u)
          fs[j] = link(j, i, link_fraction<L, T>(xs, gn, gc1[0], gc1[1], gc1[2], i));
      }
    } else {
      for (int j = 1; j < Q; j++) {
        const int i = L::opp(j);
        if (!((nb_solid >> i) & 1u)) continue;
        const T v = link(j, i, link_fraction_rt<L, T>(xs, gn, gc1[0], gc1[1], gc1[2], i));
#pragma unroll
        for (int k = 1; k < Q; k++)
          if (k == j) fs[k] = v;
      }
    }
  }
  // mirror and wall faces: specular reflection or halfway bounce-back for f
  // and every g_f (a mirror link with a solid image keeps the value above)
  // (the g_eq form is periodic only)
  // (unrolled over the directions: the crossing links' loads are in flight
  // together and each lands in a fixed register)
  if constexpr (FC) {
    if (on_wall_face(a.face, x, y, z, a.nx, a.ny, a.nz)) {
#pragma unroll
      for (int j = 1; j < Q; j++) {
        int k;
        const int cr = face_cross<L>(a.face, x, y, z, a.nx, a.ny, a.nz, j, &k);
        if (cr != 0) {
          const int src = cr == 2 ? n : h.plus_rt<L>(L::opp(j));
          const bool interp = cr == 1 && !solid_x && ((nb_solid >> L::opp(j)) & 1u);
          if (!interp) fs[j] = a.fin[k][src];
#pragma unroll
          for (int f = 0; f < NF; f++)
            gs[f][j] = plane(a.g_in + (long long)f * Q * a.pitch, a.pitch, k)[src];
        }
      }
    }
  }

  // ---- moments: rho u = sum c f + F/2, pt = sum f + u.G[rho]/2
  T u[3] = {T(0), T(0), T(0)}, pt = T(1);
  if (!solid_x) {
    // opposite directions (j, j + 1) as one pair: their sum and difference
    // in one operation, the sum into the density, the difference into the
    // momentum (c_{j+1} = -c_j)
    T m0 = fs[0], m1[3] = {T(0), T(0), T(0)};
    const Pr<T> pmj = pr(T(1), T(-1));
#pragma unroll
    for (int j = 1; j < Q; j += 2) {
      const Pr<T> sd = pr_fma(pr(fs[j + 1], fs[j + 1]), pmj, pr(fs[j], fs[j]));
      m0 += sd.a;
      if (L::cx(j)) m1[0] += T(L::cx(j)) * sd.b;
      if (L::cy(j)) m1[1] += T(L::cy(j)) * sd.b;
      if (L::cz(j)) m1[2] += T(L::cz(j)) * sd.b;
    }
    // one reciprocal per node (with equal densities, the host's)
    const T ir = RCV ? T(1) / rho : a.irho;
    for (int e = 0; e < 3; e++) u[e] = (m1[e] + T(0.5) * F[e]) * ir;
    pt = RCV ? m0 + T(0.5) * (u[0] * gR[0] + u[1] * gR[1] + u[2] * gR[2]) : m0;
  }
  if constexpr (MODE == ML_FIELDS) {
    T v;
    switch (a.field) {
      case DSM_FIELD_C1: v = cv[0]; break;
      case DSM_FIELD_C2: v = cv[1 + (a.index < NF ? a.index : NF)]; break;
      case DSM_FIELD_MU: v = mu[a.index < NF ? a.index : 0]; break;
      case DSM_FIELD_UX: v = u[0]; break;
      case DSM_FIELD_UY: v = u[1]; break;
      case DSM_FIELD_UZ: v = u[2]; break;
      case DSM_FIELD_PT: v = pt; break;
      case DSM_FIELD_RHO: v = rho; break;
      default: v = T(1) / om; break;
    }
    a.out[n] = v;
    return;
  }

  // ---- BGK collision of f (Eq. [eqn:feq], Eq. [eqn:hydroforce]) and of g_f
  {
    T chk = pt + u[0] + u[1] + u[2];
#pragma unroll
    for (int f = 0; f < NF; f++) chk += mu[f] + cv[1 + f];
    if (!isfinite(chk)) atomicOr(a.err, ERR_NONFINITE);
  }
  const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T ug = u[0] * gR[0] + u[1] * gR[1] + u[2] * gR[2];
  const T kF = T(1) - T(0.5) * om;
  {  // rest population
    const T w = T(L::w(0));
    const T s = -(T(1.5) * uu);
    T fo = w;
    if (!solid_x) {
      T Fi = T(0);
      if constexpr (RCV) Fi = kF * w * (-ug * s);
      fo = fs[0] + (w * (pt + rho * s) - fs[0]) * om + Fi;
    }
    a.fout[0][n] = fo;
    if constexpr (!EQ) {
#pragma unroll
      for (int f = 0; f < NF; f++) {
        const T Cf = cv[1 + f];
        const T geq = Cf - (T(1) - w) * mu[f] + w * Cf * s;
        T *go = a.g_out + (long long)f * Q * a.pitch;
        plane(go, a.pitch, 0)[n] = gs[f][0] + (geq - gs[f][0]) * a.omg;
      }
    }
  }
  // opposite directions (i, i + 1) as pairs: s = even +- odd (c_{i+1} = -c_i),
  // and every later operation once for both (dsm_pair.cuh)
  const Pr<T> pm = pr(T(1), T(-1)), m1 = pr(T(-1), T(-1));
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int ib = i + 1;
    const T w = T(L::w(i));
    // c_i . v over the components c_i has (cdot: no products by zero)
    const T cu = cdot<L>(i, u[0], u[1], u[2]);
    const T even = T(4.5) * cu * cu - T(1.5) * uu;
    const T odd = T(3) * cu;
    const Pr<T> s2 = pr_fma(pr(odd, odd), pm, pr(even, even));
    T fp = w, fm = w;
    if (!solid_x) {
      const T cF3 = T(3) * cdot<L>(i, F[0], F[1], F[2]);
      const T kw = kF * w;
      Pr<T> F2;
      if constexpr (RCV) {
        const T cg = cdot<L>(i, gR[0], gR[1], gR[2]);
        F2 = pr_mul(pr(kw, kw), pr_fma(pr(cg - ug, -cg - ug), s2, pr(cF3, -cF3)));
      } else {
        const T Fp = kw * cF3;
        F2 = pr(Fp, -Fp);
      }
      const Pr<T> f2 = pr(fs[i], fs[ib]);
      const Pr<T> e = pr_mul(pr(w, w), pr_fma(pr(rho, rho), s2, pr(pt, pt)));
      const Pr<T> o = pr_add(pr_fma(pr_fma(f2, m1, e), pr(om, om), f2), F2);
      fp = o.a;
      fm = o.b;
    }
    a.fout[i][n] = fp;
    a.fout[ib][n] = fm;
    if constexpr (!EQ) {
#pragma unroll
      for (int f = 0; f < NF; f++) {
        const T Cf = cv[1 + f];
        const Pr<T> geq = pr_mul(pr(w, w), pr_fma(pr(Cf, Cf), s2, pr(mu[f], mu[f])));
        const Pr<T> g2 = pr(gs[f][i], gs[f][ib]);
        const Pr<T> go = pr_fma(pr_fma(g2, m1, geq), pr(a.omg, a.omg), g2);
        T *gb = a.g_out + (long long)f * Q * a.pitch;
        plane(gb, a.pitch, i)[n] = go.a;
        plane(gb, a.pitch, ib)[n] = go.b;
      }
    }
  }
  if constexpr (EQ) {
    // g* = g_eq (tau_g = 1): store what fixes it
    T Af[NF], Cf[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) {
      Af[f] = mu[f] - T(1.5) * cv[1 + f] * uu;
      Cf[f] = cv[1 + f];
    }
    io.template put_eq<L, NF>(a, n, Af, Cf, u);
  }
}

template <int K, class T, int NF, int MODE, bool EQ, bool FC, bool RCV = true>
__global__ void __launch_bounds__(256) ml_node_kernel(MLArgs<T> a) {
  ml_node_body<K, T, NF, MODE, EQ, FC, MLGlobalIO<T>, RCV>(
      a, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y,
      blockIdx.z * blockDim.z + threadIdx.z);
}
// D3Q19 FP32 with three free fluids and a mirror or wall face: the unrolled
// face fix-ups raise the register count past one 256-thread block per SM, and
// asking for two (128 registers, no spills) ran 12 % faster.  With fewer free
// fluids the cap was slower, so those keep the plain kernel.
template <int K, class T, int NF, int MODE>
__global__ void __launch_bounds__(256, 2) ml_node_faces_kernel(MLArgs<T> a) {
  ml_node_body<K, T, NF, MODE, false, true>(a, blockIdx.x * blockDim.x + threadIdx.x,
                                           blockIdx.y * blockDim.y + threadIdx.y,
                                           blockIdx.z * blockDim.z + threadIdx.z);
}
template <int K, class T, int NF>
constexpr bool ml_faces_capped() {
  return K == 1 && sizeof(T) == 4 && NF >= 3;
}

// initial state at rest: f_i = w_i, g_f,i = g_eq,i(C_f, mu_f(C), u = 0); C
// (NF planes) is read from a.C
template <int K, class T, int NF, bool EQ>
__global__ void __launch_bounds__(256) ml_init_kernel(MLArgs<T> a) {
  using L = Lat<K>;
  constexpr int Q = L::Q;
  constexpr int NC = NF + 2;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x >= a.nx || y >= a.ny || z >= a.nz) return;
  Hood h;
  h.init_faces(x, y, z, a.nx, a.ny, a.nz, a.face);
  h.guard(a.err);
  const int n = h.g(h.ox[1] + h.oy[1] + h.oz[1]);
  T cv[NC], lap[NC];
  cv[0] = a.C1[n];
  T last = T(1) - cv[0];
  for (int f = 0; f < NF; f++) {
    cv[1 + f] = a.C[f * a.pitch + n];
    last -= cv[1 + f];
  }
  cv[NC - 1] = last;
  for (int k = 0; k < NC; k++) lap[k] = T(0);
  for (int i = 1; i < Q; i++) {
    const int m = h.plus_rt<L>(i);
    const T w = T(L::w(i));
    const T c1m = a.C1[m];
    T lastm = T(1) - c1m;
    for (int f = 0; f < NF; f++) {
      const T cm = a.C[f * a.pitch + m];
      lastm -= cm;
      lap[1 + f] += w * (cm - cv[1 + f]);
    }
    lap[0] += w * (c1m - cv[0]);
    lap[NC - 1] += w * (lastm - cv[NC - 1]);
  }
  T d[NC];
  for (int k = 0; k < NC; k++)
    d[k] = a.kappa[k] * bwell(cv[k]) - a.a2 * a.kappa[k] * (T(6) * lap[k]);
  for (int i = 0; i < Q; i++) {
    const T w = T(L::w(i));
    plane(a.f_out, a.pitch, i)[n] = w;
    if constexpr (!EQ) {
      for (int f = 0; f < NF; f++) {
        const T mu = d[1 + f] - d[NC - 1];
        const T Cf = cv[1 + f];
        T *go = a.g_out + (long long)f * Q * a.pitch;
        plane(go, a.pitch, i)[n] = i == 0 ? Cf - (T(1) - w) * mu : w * mu;
      }
    }
  }
  if constexpr (EQ) {  // at rest: A_f = mu_f, u = 0
    for (int f = 0; f < NF; f++) a.A[f * a.pitch + n] = d[1 + f] - d[NC - 1];
    for (int e = 0; e < L::D; e++) a.U[e * a.pitch + n] = T(0);
  }
}

// the populations of g held as g_eq, for reading the state: g_f,i(x) =
// g_eq_i(A_f, C_f, u at x), C_f that of the state's last collision; dense
// output, NF blocks of Q rows of N
template <int K, class T, int NF>
__global__ void __launch_bounds__(256) ml_g_of_eq_kernel(MLArgs<T> a, T *out) {
  using L = Lat<K>;
  constexpr int Q = L::Q;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N;
       n += (long long)gridDim.x * blockDim.x) {
    const T ux = a.U[n], uy = a.U[a.pitch + n], uz = L::D == 3 ? a.U[2 * a.pitch + n] : T(0);
    const T uu = ux * ux + uy * uy + uz * uz;
    for (int f = 0; f < NF; f++) {
      const T A = a.A[f * a.pitch + n], Cf = a.Cprev[f * a.pitch + n];
      for (int i = 0; i < Q; i++) {
        const T v = i == 0 ? Cf - T(1.0 - L::w(0)) * A - T(1.5) * Cf * uu
                           : T(L::w(i)) * geq_core(A, Cf, cdot<L>(i, ux, uy, uz));
        out[((long long)f * Q + i) * a.N + n] = v;
      }
    }
  }
}

}  // namespace dsm

#include "dsm_mlz.cuh"

using namespace dsm;

struct dsm_mlattice {
  dsm_params prm;
  int nf, q, real_bytes;
  double kappa[ML_MAX_NF + 2], rho[ML_MAX_NF + 1], tau[ML_MAX_NF + 1];
  long long N, pitch;
  cudaStream_t stream;
  char *f[2], *g[2], *C[2], *C1, *M;  // C[cur]: C of the last collision; M: A_f and u
  int *err;                            // latched error word in the workspace
  int cur;
  bool eq;  // g held as g_eq (tau_g = 1, periodic faces)
  bool has_solid, has_fluid;
  // single-pass step (dsm_mlz.cuh): eligible lattice, state held in the padded
  // buffers (zc: the current one), tensor maps per buffer (quads, u_z, pairs, C1)
  bool zok, zpacked, zmaps_ok;
  int zc, nxp, nyp, step_form, zrun, zrun_auto;
  char *Qz[2], *Uz[2], *Pz[2], *C1z;
  CUtensorMap maps[2][4];
};

namespace {

struct MLLayout {
  size_t f[2], g[2], C[2], C1, M, err, Qz[2], Uz[2], Pz[2], C1z, total;
};

// g held as g_eq: tau_g = 1 and every face periodic
bool ml_eq(const dsm_params *p) { return p->tau_g == 1.0 && !has_walls(p); }

// the single-pass step applies: D3Q19, g held as g_eq, at least one 32 x 8
// tile (the last tiles may be ragged)
bool ml_z_eligible(const dsm_params *p) {
  return p->lattice == DSM_D3Q19 && ml_eq(p) && z_tiles(p->nx, p->ny);
}

MLLayout ml_layout(int q, int nf, int real_bytes, long long pitch, bool eq,
                   const dsm_params *p = nullptr) {
  MLLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (size_t)round_up((long long)bytes, 256);
    return at;
  };
  for (int b = 0; b < 2; b++) L.f[b] = take((size_t)q * pitch * real_bytes);
  for (int b = 0; b < 2; b++) L.g[b] = take(eq ? 0 : (size_t)nf * q * pitch * real_bytes);
  for (int b = 0; b < 2; b++) L.C[b] = take((size_t)nf * pitch * real_bytes);
  L.C1 = take((size_t)pitch * real_bytes);
  L.M = take(eq ? (size_t)(nf + 3) * pitch * real_bytes : 0);
  L.err = take(sizeof(int));
  // padded buffers of the single-pass step: per padded node a quad, u_z and
  // nf - 1 pairs (two buffers), and C1
  const bool z = p && ml_z_eligible(p);
  const size_t P = z ? (size_t)z_padded_x(p->nx) * z_padded_y(p->ny) * p->nz : 0;
  for (int b = 0; b < 2; b++) {
    L.Qz[b] = take(4 * P * real_bytes);
    L.Uz[b] = take(P * real_bytes);
    L.Pz[b] = take(2 * (size_t)(nf - 1) * P * real_bytes);
  }
  L.C1z = take(P * real_bytes);
  L.total = o;
  return L;
}

dsm_status ml_check(const dsm_params *p, int nfluid, const double *kappa, const double *rho,
                    const double *tau) {
  if (!p || !kappa || !rho || !tau) return DSM_E_INVAL;
  if (p->lattice != DSM_D2Q9 && p->lattice != DSM_D3Q19) return DSM_E_INVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->lattice == DSM_D2Q9 && p->nz != 1))
    return DSM_E_INVAL;
  if ((long long)p->nx * p->ny * p->nz >= (1ll << 31)) return DSM_E_INVAL;
  if (nfluid < 2 || nfluid > ML_MAX_NF + 1) return DSM_E_INVAL;
  if (!(p->alpha > 0.0) || p->alpha_s < 0.0 || !(p->tau_g > 0.5)) return DSM_E_INVAL;
  if (!faces_valid(p)) return DSM_E_INVAL;
  for (int k = 0; k <= nfluid; k++)
    if (!isfinite(kappa[k]) || (k > 0 && !(kappa[k] > 0.0))) return DSM_E_INVAL;
  for (int f = 0; f < nfluid; f++)
    if (!(rho[f] > 0.0) || !(tau[f] > 0.5)) return DSM_E_INVAL;
  if (p->precision != DSM_F64 && p->precision != DSM_F32) return DSM_E_UNSUPPORTED;
  return DSM_OK;
}

template <class T>
MLArgs<T> ml_args(const dsm_mlattice *h, int src) {
  MLArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.nx = h->prm.nx;
  a.ny = h->prm.ny;
  a.nz = h->prm.nz;
  a.N = h->N;
  a.pitch = h->pitch;
  for (int k = 0; k < 6; k++) {
    a.face[k] = h->prm.face[k];
    a.walls |= h->prm.face[k] != 0;
  }
  for (int k = 0; k <= h->nf + 1; k++) a.kappa[k] = T(h->kappa[k]);
  for (int f = 0; f <= h->nf; f++) {
    a.rho[f] = T(h->rho[f]);
    a.om[f] = T(1.0 / h->tau[f]);
  }
  a.omg = T(1.0 / h->prm.tau_g);
  a.irho = T(1.0 / h->rho[h->nf]);
  for (int f = 0; f < h->nf; f++) a.rc |= h->rho[f] != h->rho[h->nf];
  a.a2 = T(h->prm.alpha * h->prm.alpha);
  a.alpha_s = T(h->prm.alpha_s > 0.0 ? h->prm.alpha_s : h->prm.alpha);
  for (int e = 0; e < 3; e++) a.body[e] = T(h->prm.body_force[e]);
  if (h->prm.lattice == DSM_D2Q9) a.body[2] = T(0);
  a.f_in = (const T *)h->f[src];
  a.g_in = (const T *)h->g[src];
  a.f_out = (T *)h->f[src ^ 1];
  for (int j = 0; j < h->q; j++) {
    a.fin[j] = a.f_in + (long long)j * a.pitch;
    a.fout[j] = a.f_out + (long long)j * a.pitch;
  }
  a.g_out = (T *)h->g[src ^ 1];
  a.C = (T *)h->C[src ^ 1];
  a.Cprev = (const T *)h->C[src];
  a.A = (T *)h->M;
  a.U = h->M ? (T *)h->M + (long long)h->nf * h->pitch : nullptr;
  a.C1 = (const T *)h->C1;
  a.err = h->err;
  a.nxp = h->nxp;
  a.nyp = h->nyp;
  if (h->zok) {  // the single-pass step writes the other padded buffer
    a.Qz = (T *)h->Qz[h->zc ^ 1];
    a.Uz = (T *)h->Uz[h->zc ^ 1];
    a.Pz = (T *)h->Pz[h->zc ^ 1];
  }
  return a;
}

dim3 ml_block(const dsm_mlattice *h) {
  return lb_block(h->prm.lattice, h->prm.nx, h->prm.ny, h->prm.nz);
}
dim3 ml_grid(const dsm_mlattice *h) {
  return lb_grid_of(ml_block(h), h->prm.nx, h->prm.ny, h->prm.nz);
}

// kernel dispatch over (lattice, free fluids) for one arithmetic type
template <class T, template <int, class, int> class Launch>
cudaError_t ml_dispatch(const dsm_mlattice *h, const MLArgs<T> &a, void *extra = nullptr) {
  const int key = h->prm.lattice * 4 + h->nf;
  const dim3 g = ml_grid(h), b = ml_block(h);
  const bool eq = h->eq;
  switch (key) {
    case 1: Launch<0, T, 1>::go(g, b, a, h->stream, eq, extra); break;
    case 2: Launch<0, T, 2>::go(g, b, a, h->stream, eq, extra); break;
    case 3: Launch<0, T, 3>::go(g, b, a, h->stream, eq, extra); break;
    case 5: Launch<1, T, 1>::go(g, b, a, h->stream, eq, extra); break;
    case 6: Launch<1, T, 2>::go(g, b, a, h->stream, eq, extra); break;
    case 7: Launch<1, T, 3>::go(g, b, a, h->stream, eq, extra); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// D3Q19 with g held as g_eq: the two-fluid z-marching tiled moments pass,
// once per free fluid, on that fluid's (A_f, C_f) planes and the shared u
// (the same per-node arithmetic as ml_moments_eq_kernel)
template <class T>
void ml_moments_eq_tiled(const MLArgs<T> &a, int nf, cudaStream_t s) {
  const size_t smem = moments_eq_smem<T>();
  if (smem > 48 * 1024) {
    static bool opted_in = false;
    if (!opted_in) {
      if (cudaFuncSetAttribute(moments_eq_tiled_kernel<T, T>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
        return;
      opted_in = true;
    }
  }
  const int tiles = ((a.nx + MT_X - 1) / MT_X) * ((a.ny + MT_Y - 1) / MT_Y);
  int zrun = 32;
  while (zrun > 4 && (long long)tiles * ((a.nz + zrun - 1) / zrun) < 6 * 152) zrun /= 2;
  const dim3 grid((a.nx + MT_X - 1) / MT_X, (a.ny + MT_Y - 1) / MT_Y, (a.nz + zrun - 1) / zrun);
  for (int f = 0; f < nf; f++) {
    LBArgs<T, T> b;
    memset(&b, 0, sizeof(b));
    b.nx = a.nx;
    b.ny = a.ny;
    b.nz = a.nz;
    b.N = a.N;
    b.pitch = a.pitch;
    b.Mp[0] = a.A + (long long)f * a.pitch;
    b.Mp[1] = a.U;
    b.Mp[2] = a.U + a.pitch;
    b.Mp[3] = a.U + 2 * a.pitch;
    b.Cprev = a.Cprev + (long long)f * a.pitch;
    b.C = a.C + (long long)f * a.pitch;
    moments_eq_tiled_kernel<T, T><<<grid, dim3(MT_X, MT_Y, 1), smem, s>>>(b, zrun);
  }
}

template <int K, class T, int NF>
struct MomentsL {
  static void go(dim3 g, dim3 b, const MLArgs<T> &a, cudaStream_t s, bool eq, void *) {
    if (eq && K == 1) ml_moments_eq_tiled<T>(a, NF, s);
    else if (eq) ml_moments_eq_kernel<K, T, NF><<<g, b, 0, s>>>(a);
    else if (a.walls) ml_moments_kernel<K, T, NF, true><<<g, b, 0, s>>>(a);
    else ml_moments_kernel<K, T, NF, false><<<g, b, 0, s>>>(a);
  }
};
template <int K, class T, int NF>
struct StepL {
  static void go(dim3 g, dim3 b, const MLArgs<T> &a, cudaStream_t s, bool eq, void *) {
    if (eq && a.rc) ml_node_kernel<K, T, NF, ML_STEP, true, false><<<g, b, 0, s>>>(a);
    else if (eq) ml_node_kernel<K, T, NF, ML_STEP, true, false, false><<<g, b, 0, s>>>(a);
    else if (!a.walls) ml_node_kernel<K, T, NF, ML_STEP, false, false><<<g, b, 0, s>>>(a);
    else if constexpr (ml_faces_capped<K, T, NF>()) ml_node_faces_kernel<K, T, NF, ML_STEP><<<g, b, 0, s>>>(a);
    else ml_node_kernel<K, T, NF, ML_STEP, false, true><<<g, b, 0, s>>>(a);
  }
};
template <int K, class T, int NF>
struct FieldsL {
  static void go(dim3 g, dim3 b, const MLArgs<T> &a, cudaStream_t s, bool eq, void *) {
    if (eq) ml_node_kernel<K, T, NF, ML_FIELDS, true, false><<<g, b, 0, s>>>(a);
    else if (!a.walls) ml_node_kernel<K, T, NF, ML_FIELDS, false, false><<<g, b, 0, s>>>(a);
    else if constexpr (ml_faces_capped<K, T, NF>()) ml_node_faces_kernel<K, T, NF, ML_FIELDS><<<g, b, 0, s>>>(a);
    else ml_node_kernel<K, T, NF, ML_FIELDS, false, true><<<g, b, 0, s>>>(a);
  }
};
template <int K, class T, int NF>
struct InitL {
  static void go(dim3 g, dim3 b, const MLArgs<T> &a, cudaStream_t s, bool eq, void *) {
    if (eq) ml_init_kernel<K, T, NF, true><<<g, b, 0, s>>>(a);
    else ml_init_kernel<K, T, NF, false><<<g, b, 0, s>>>(a);
  }
};
template <int K, class T, int NF>
struct GofEqL {
  static void go(dim3, dim3, const MLArgs<T> &a, cudaStream_t s, bool, void *out) {
    long long blocks = (a.N + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    ml_g_of_eq_kernel<K, T, NF><<<(int)blocks, 256, 0, s>>>(a, (T *)out);
  }
};

// ---- single-pass step --------------------------------------------------------
template <class T, int NF>
struct MLZ {
  static bool prepare() {  // opt in to the kernels' dynamic shared memory, once
    static const bool ok =
        cudaFuncSetAttribute(mlz_kernel<T, NF, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)MLZSmem<T, NF>::total) == cudaSuccess &&
        cudaFuncSetAttribute(mlz_kernel<T, NF, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)MLZSmem<T, NF>::total) == cudaSuccess;
    return ok;
  }
  static int resident() {
    int b = 0;
    if (!prepare() || cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                          &b, mlz_kernel<T, NF, true>, ZT_X * ZT_Y, MLZSmem<T, NF>::total) !=
                          cudaSuccess)
      return 0;
    return b;
  }
  static cudaError_t step(const MLArgs<T> &a, const CUtensorMap *m, int zrun, cudaStream_t s) {
    if (!prepare()) return cudaErrorInvalidValue;
    const dim3 grid(z_tiles_x(a.nx), z_tiles_y(a.ny), (a.nz + zrun - 1) / zrun),
        blk(ZT_X, ZT_Y, 1);
    if (a.rc)
      mlz_kernel<T, NF, true><<<grid, blk, MLZSmem<T, NF>::total, s>>>(a, zrun, m[0], m[1], m[2], m[3]);
    else
      mlz_kernel<T, NF, false><<<grid, blk, MLZSmem<T, NF>::total, s>>>(a, zrun, m[0], m[1], m[2], m[3]);
    return cudaGetLastError();
  }
  static cudaError_t pack(const MLArgs<T> &a, dsm_mlattice *h, cudaStream_t s) {
    mlz_pack_kernel<T, NF><<<152 * 8, 256, 0, s>>>(a, (T *)h->Qz[0], (T *)h->Qz[1], (T *)h->Uz[0],
                                                   (T *)h->Uz[1], (T *)h->Pz[0], (T *)h->Pz[1],
                                                   (T *)h->C1z);
    return cudaGetLastError();
  }
  static cudaError_t unpack(const MLArgs<T> &a, dsm_mlattice *h, T *Cout, cudaStream_t s) {
    mlz_unpack_kernel<T, NF><<<152 * 8, 256, 0, s>>>(a, (const T *)h->Qz[h->zc],
                                                     (const T *)h->Uz[h->zc],
                                                     (const T *)h->Pz[h->zc], Cout);
    return cudaGetLastError();
  }
};

// dispatch over the free fluids of a D3Q19 lattice
template <class T, class Fn>
cudaError_t mlz_dispatch(const dsm_mlattice *h, Fn fn) {
  switch (h->nf) {
    case 1: return fn(MLZ<T, 1>());
    case 2: return fn(MLZ<T, 2>());
    case 3: return fn(MLZ<T, 3>());
    default: return cudaErrorInvalidValue;
  }
}

bool mlz_maps(dsm_mlattice *h) {
  if (h->zmaps_ok) return true;
  const int rb = h->real_bytes, nz = h->prm.nz;
  for (int b = 0; b < 2; b++) {
    CUtensorMap *m = h->maps[b];
    if (!encode_plane_map(&m[0], h->Qz[b], rb, 4, h->nxp, h->nyp, nz, ZB_Y) ||
        !encode_plane_map(&m[1], h->Uz[b], rb, 1, h->nxp, h->nyp, nz, ZB_Y) ||
        !encode_plane_map(&m[3], h->C1z, rb, 1, h->nxp, h->nyp, nz, ZB1_Y))
      return false;
    if (h->nf > 1) {
      if (!encode_plane_map(&m[2], h->Pz[b], rb, 2, h->nxp, h->nyp, (h->nf - 1) * nz, ZB_Y))
        return false;
    } else {
      m[2] = m[0];  // no pairs: never loaded
    }
  }
  h->zmaps_ok = true;
  return true;
}

// planes per block: the same wave model as the two-fluid single-pass step
// (runs of zr planes in waves of the resident blocks, each run paying about
// 0.7 of a plane for its prologue)
template <class T>
int mlz_auto_run(dsm_mlattice *h) {
  if (h->zrun_auto) return h->zrun_auto;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 0;
  mlz_dispatch<T>(h, [&](auto k) {
    per_sm = k.resident();
    return cudaSuccess;
  });
  const long long resident = (long long)(sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
  const long long tiles = (long long)z_tiles_x(h->prm.nx) * z_tiles_y(h->prm.ny);
  const int nz = h->prm.nz;
  double best = 1e300;
  int run = nz;
  for (int zr = 1; zr <= nz; zr++) {
    const long long blocks = tiles * ((nz + zr - 1) / zr);
    const double waves = (double)((blocks + resident - 1) / resident);
    const double cost = waves * (zr + 0.7);
    if (cost < best - 1e-9) {
      best = cost;
      run = zr;
    }
  }
  h->zrun_auto = run;
  return run;
}

bool mlz_active(const dsm_mlattice *h) { return h->zok && h->step_form == DSM_STEP_AUTO; }

// padded state -> canonical state, before anything reads the canonical layout
template <class T>
cudaError_t mlz_unpack(dsm_mlattice *h) {
  if (!h->zpacked) return cudaSuccess;
  const MLArgs<T> a = ml_args<T>(h, h->cur);
  T *Cout = (T *)h->C[h->cur];
  const cudaError_t e = mlz_dispatch<T>(h, [&](auto k) { return k.unpack(a, h, Cout, h->stream); });
  if (e == cudaSuccess) h->zpacked = false;
  return e;
}

template <class T>
cudaError_t ml_step(dsm_mlattice *h) {
  if (mlz_active(h)) {
    if (!h->zpacked) {
      if (!mlz_maps(h)) return cudaErrorInvalidValue;
      const MLArgs<T> a = ml_args<T>(h, h->cur);
      const cudaError_t e = mlz_dispatch<T>(h, [&](auto k) { return k.pack(a, h, h->stream); });
      if (e != cudaSuccess) return e;
      h->zc = 0;
      h->zpacked = true;
    }
    const MLArgs<T> a = ml_args<T>(h, h->cur);
    const int zrun = h->zrun > 0 ? h->zrun : mlz_auto_run<T>(h);
    const CUtensorMap *m = h->maps[h->zc];
    const cudaError_t e =
        mlz_dispatch<T>(h, [&](auto k) { return k.step(a, m, zrun, h->stream); });
    if (e == cudaSuccess) {
      h->zc ^= 1;
      h->cur ^= 1;
    }
    return e;
  }
  cudaError_t e = mlz_unpack<T>(h);
  if (e != cudaSuccess) return e;
  MLArgs<T> a = ml_args<T>(h, h->cur);
  e = ml_dispatch<T, MomentsL>(h, a);
  if (e == cudaSuccess) e = ml_dispatch<T, StepL>(h, a);
  if (e == cudaSuccess) h->cur ^= 1;
  return e;
}

template <class T>
cudaError_t ml_fields(dsm_mlattice *h, int field, int index, void *dst) {
  const cudaError_t eu = mlz_unpack<T>(h);
  if (eu != cudaSuccess) return eu;
  MLArgs<T> a = ml_args<T>(h, h->cur);
  a.field = field;
  a.index = index;
  a.out = (T *)dst;
  cudaError_t e = ml_dispatch<T, MomentsL>(h, a);
  if (e == cudaSuccess) e = ml_dispatch<T, FieldsL>(h, a);
  return e;
}

dsm_status ml_status(cudaError_t e) { return e == cudaSuccess ? DSM_OK : DSM_E_CUDA; }

}  // namespace

extern "C" {

dsm_status dsm_ml_workspace_bytes(const dsm_params *p, int nfluid, size_t *bytes) {
  if (!p || !bytes) return DSM_E_INVAL;
  if (p->lattice != DSM_D2Q9 && p->lattice != DSM_D3Q19) return DSM_E_INVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || nfluid < 2 || nfluid > ML_MAX_NF + 1)
    return DSM_E_INVAL;
  if (p->precision != DSM_F64 && p->precision != DSM_F32) return DSM_E_UNSUPPORTED;
  const long long N = (long long)p->nx * p->ny * p->nz;
  const int q = p->lattice == DSM_D2Q9 ? 9 : 19;
  *bytes = ml_layout(q, nfluid - 1, p->precision == DSM_F64 ? 8 : 4, round_up(N, 64), ml_eq(p), p)
               .total;
  return DSM_OK;
}

dsm_status dsm_ml_create(const dsm_params *p, int nfluid, const double *kappa, const double *rho,
                         const double *tau, void *d_workspace, size_t bytes, void *cuda_stream,
                         dsm_mlattice **out) {
  if (!out) return DSM_E_INVAL;
  *out = nullptr;
  dsm_status s = ml_check(p, nfluid, kappa, rho, tau);
  if (s != DSM_OK) return s;
  const long long N = (long long)p->nx * p->ny * p->nz;
  const long long pitch = round_up(N, 64);
  const int q = p->lattice == DSM_D2Q9 ? 9 : 19;
  const int rb = p->precision == DSM_F64 ? 8 : 4;
  const MLLayout L = ml_layout(q, nfluid - 1, rb, pitch, ml_eq(p), p);
  if (!d_workspace || bytes < L.total || ((uintptr_t)d_workspace & 255u)) return DSM_E_WORKSPACE;
  dsm_mlattice *h = new (std::nothrow) dsm_mlattice;
  if (!h) return DSM_E_INVAL;
  memset(h, 0, sizeof(*h));
  h->prm = *p;
  h->nf = nfluid - 1;
  h->q = q;
  h->real_bytes = rb;
  for (int k = 0; k <= nfluid; k++) h->kappa[k] = kappa[k];
  for (int f = 0; f < nfluid; f++) {
    h->rho[f] = rho[f];
    h->tau[f] = tau[f];
  }
  h->N = N;
  h->pitch = pitch;
  h->stream = (cudaStream_t)cuda_stream;
  h->eq = ml_eq(p);
  char *w = (char *)d_workspace;
  for (int b = 0; b < 2; b++) {
    h->f[b] = w + L.f[b];
    h->g[b] = h->eq ? nullptr : w + L.g[b];
    h->C[b] = w + L.C[b];
  }
  h->C1 = w + L.C1;
  h->M = h->eq ? w + L.M : nullptr;
  h->err = (int *)(w + L.err);
  h->zok = ml_z_eligible(p);
  h->nxp = z_padded_x(p->nx);
  h->nyp = z_padded_y(p->ny);
  for (int b = 0; b < 2 && h->zok; b++) {
    h->Qz[b] = w + L.Qz[b];
    h->Uz[b] = w + L.Uz[b];
    h->Pz[b] = w + L.Pz[b];
  }
  h->C1z = h->zok ? w + L.C1z : nullptr;
  // no solid until one is set: C1 = 0; no error latched
  if (cudaMemsetAsync(h->C1, 0, (size_t)pitch * rb, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->err, 0, sizeof(int), h->stream) != cudaSuccess) {
    delete h;
    return DSM_E_CUDA;
  }
  *out = h;
  return DSM_OK;
}

dsm_status dsm_ml_set_solid(dsm_mlattice *h, const void *d_field, int kind) {
  if (!h || !d_field || (kind != 0 && kind != 1)) return DSM_E_INVAL;
  cudaError_t e;
  if (kind == 1) {
    e = cudaMemcpyAsync(h->C1, d_field, (size_t)h->N * h->real_bytes, cudaMemcpyDeviceToDevice,
                        h->stream);
  } else {
    long long blocks = (h->N + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const double as = h->prm.alpha_s > 0.0 ? h->prm.alpha_s : h->prm.alpha;
    if (h->real_bytes == 8)
      solid_profile_kernel<double><<<(int)blocks, 256, 0, h->stream>>>(
          (const double *)d_field, (double *)h->C1, h->N, as);
    else
      solid_profile_kernel<float><<<(int)blocks, 256, 0, h->stream>>>(
          (const float *)d_field, (float *)h->C1, h->N, (float)as);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return DSM_E_CUDA;
  h->has_solid = true;
  h->has_fluid = false;
  h->zpacked = false;
  return DSM_OK;
}

dsm_status dsm_ml_set_fluids(dsm_mlattice *h, const void *d_c) {
  if (!h || !d_c) return DSM_E_INVAL;
  // the free fluids into C[0] (plane by plane), then the rest state into
  // buffer 0 (with g held as g_eq, C[0] is then the C of the state)
  for (int f = 0; f < h->nf; f++) {
    cudaError_t e = cudaMemcpyAsync(h->C[0] + (size_t)f * h->pitch * h->real_bytes,
                                    (const char *)d_c + (size_t)f * h->N * h->real_bytes,
                                    (size_t)h->N * h->real_bytes, cudaMemcpyDeviceToDevice,
                                    h->stream);
    if (e != cudaSuccess) return DSM_E_CUDA;
  }
  h->cur = 0;
  h->zpacked = false;
  if (cudaMemsetAsync(h->err, 0, sizeof(int), h->stream) != cudaSuccess) return DSM_E_CUDA;
  cudaError_t e;
  if (h->real_bytes == 8) e = ml_dispatch<double, InitL>(h, ml_args<double>(h, 1));
  else e = ml_dispatch<float, InitL>(h, ml_args<float>(h, 1));
  if (e != cudaSuccess) return DSM_E_CUDA;
  h->has_fluid = true;
  return DSM_OK;
}

dsm_status dsm_ml_step(dsm_mlattice *h, long long nsteps) {
  TraceRange trace_range("N-fluid step");
  if (!h || nsteps < 0) return DSM_E_INVAL;
  if (!h->has_fluid) return DSM_E_STATE;
  for (long long t = 0; t < nsteps; t++) {
    const cudaError_t e = h->real_bytes == 8 ? ml_step<double>(h) : ml_step<float>(h);
    if (e != cudaSuccess) return DSM_E_CUDA;
  }
  return DSM_OK;
}

dsm_status dsm_ml_get_field(dsm_mlattice *h, int field, int index, void *d_dst) {
  if (!h || !d_dst || field < DSM_FIELD_C1 || field > DSM_FIELD_TAU) return DSM_E_INVAL;
  if (field == DSM_FIELD_C3) return DSM_E_INVAL;
  if (field == DSM_FIELD_C2 && (index < 0 || index > h->nf)) return DSM_E_INVAL;
  if (field == DSM_FIELD_MU && (index < 0 || index >= h->nf)) return DSM_E_INVAL;
  if (!h->has_fluid) return DSM_E_STATE;
  return ml_status(h->real_bytes == 8 ? ml_fields<double>(h, field, index, d_dst)
                                      : ml_fields<float>(h, field, index, d_dst));
}

dsm_status dsm_ml_get_populations(dsm_mlattice *h, void *d_f, void *d_g) {
  if (!h || (!d_f && !d_g)) return DSM_E_INVAL;
  if (!h->has_fluid) return DSM_E_STATE;
  const size_t row = (size_t)h->N * h->real_bytes, pb = (size_t)h->pitch * h->real_bytes;
  for (int i = 0; d_f && i < h->q; i++)
    if (cudaMemcpyAsync((char *)d_f + i * row, h->f[h->cur] + i * pb, row,
                        cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
      return DSM_E_CUDA;
  if (d_g && h->eq) {  // rebuilt from (A_f, C_f, u)
    const cudaError_t eu = h->real_bytes == 8 ? mlz_unpack<double>(h) : mlz_unpack<float>(h);
    if (eu != cudaSuccess) return DSM_E_CUDA;
    const cudaError_t e = h->real_bytes == 8
                              ? ml_dispatch<double, GofEqL>(h, ml_args<double>(h, h->cur), d_g)
                              : ml_dispatch<float, GofEqL>(h, ml_args<float>(h, h->cur), d_g);
    return e == cudaSuccess ? DSM_OK : DSM_E_CUDA;
  }
  for (int i = 0; d_g && i < h->nf * h->q; i++)
    if (cudaMemcpyAsync((char *)d_g + i * row, h->g[h->cur] + i * pb, row,
                        cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
      return DSM_E_CUDA;
  return DSM_OK;
}

dsm_status dsm_ml_check(dsm_mlattice *h) {
  if (!h) return DSM_E_INVAL;
  int word = 0;
  if (cudaMemcpyAsync(&word, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return DSM_E_CUDA;
  if (word & ERR_TIMEOUT) return DSM_E_TIMEOUT;
  if (word & ERR_BOUNDS) return DSM_E_BOUNDS;
  return (word & ERR_NONFINITE) ? DSM_E_NONFINITE : DSM_OK;
}

dsm_status dsm_ml_set_step_form(dsm_mlattice *h, int form, int zrun) {
  if (!h || (form != DSM_STEP_AUTO && form != DSM_STEP_TWO_PASS) || zrun < 0) return DSM_E_INVAL;
  h->step_form = form;
  h->zrun = zrun;
  return DSM_OK;
}

dsm_status dsm_ml_step_info(dsm_mlattice *h, int *single_pass, int *zrun) {
  if (!h) return DSM_E_INVAL;
  const bool single = mlz_active(h);
  if (single_pass) *single_pass = single ? 1 : 0;
  if (zrun) {
    *zrun = 0;
    if (single) *zrun = h->zrun > 0 ? h->zrun
                                    : (h->real_bytes == 8 ? mlz_auto_run<double>(h)
                                                          : mlz_auto_run<float>(h));
  }
  return DSM_OK;
}

dsm_status dsm_ml_destroy(dsm_mlattice *h) {
  delete h;
  return DSM_OK;
}

}  // extern "C"
