// dsm_lb_impl.cuh -- lattice Boltzmann kernels of the Diffuse Solid Method
// (Sec. II.B of the paper), templated on lattice (D2Q9 / D3Q19), arithmetic
// type T and population storage type S.  Each dsm_lb_<precision>.cu includes
// this file and instantiates one storage type.
//
// State: POST-COLLISION populations f*, g* in two ping-pong buffers,
// structure-of-arrays (plane i at offset i*pitch).  One step =
//   moments pass   C(x) = sum_i g*_i(x - c_i)                       (K1)
//   fused pass     pull f, g (interpolated bounce-back at the diffuse solid),
//                  mu, forces, moments, BGK collision of f and g     (K2)
// The fused pass needs C and C1 on the node's 1-neighbourhood only, because
// the capillary force is taken in its potential form mu G[C] (see below).
//
// g held as g_eq.  With tau_g = 1 the g collision replaces g_i by g_eq_i
// entirely, and g_eq_i depends on the node's C, mu and u only.  The fused pass
// then stores A = mu - 3/2 C u.u and u instead of the Q populations, and the
// moments pass rebuilds C(x) = sum_i g_eq_i(x - c_i) from the neighbours'
// (A, C, u): for i != 0, g_eq_i = w_i (A + C c_i.u (3 + 9/2 c_i.u)), and the
// rest population holds the remainder C - (1 - w_0) A - 3/2 C u.u.  Same
// trajectory, up to rounding; 4 + 1 reals per node move instead of 2Q.
#pragma once

#include <vector>

#include "dsm_common.cuh"
#include "dsm_pair.cuh"
#include "dsm_reduce.cuh"

namespace dsm {

enum { MODE_STEP = 0, MODE_FIELDS = 1, MODE_OBS = 2 };
constexpr int OBS_K = 5;  // sum C, sum C1, kinetic, max |u|, nonfinite

template <class T>
__device__ __forceinline__ T bwell(T c) {
  // d/dc [c^2 (1-c)^2 / 2] = c (1 - c)(1 - 2c)   (Sec. II.B)
  return c * (T(1) - c) * (T(1) - T(2) * c);
}

// Periodic neighbourhood of node (x, y, z): linear index of x + c.  (Host-
// callable: the CPU tests check its indices against the wrapped coordinates.)
struct Hood {
  int ox[3], oy[3], oz[3];
#ifdef DSM_CHECKED
  // checked build: the neighbour indices are guarded against the lattice
  // (chk, dsm_common.cuh); guard() names the error word to latch
  int *err = nullptr;
  long long lim = 0;
  __host__ __device__ __forceinline__ void guard(int *e) { err = e; }
  __host__ __device__ __forceinline__ int g(int v) const { return chk(err, v, lim); }
#else
  __host__ __device__ __forceinline__ void guard(int *) {}
  __host__ __device__ __forceinline__ int g(int v) const { return v; }
#endif
  __host__ __device__ __forceinline__ void init(int x, int y, int z, int nx, int ny, int nz) {
#ifdef DSM_CHECKED
    lim = (long long)nx * ny * nz;
#endif
    ox[0] = x == 0 ? nx - 1 : x - 1;
    ox[1] = x;
    ox[2] = x + 1 == nx ? 0 : x + 1;
    int ym = y == 0 ? ny - 1 : y - 1, yp = y + 1 == ny ? 0 : y + 1;
    oy[0] = ym * nx;
    oy[1] = y * nx;
    oy[2] = yp * nx;
    int zm = z == 0 ? nz - 1 : z - 1, zp = z + 1 == nz ? 0 : z + 1;
    const int s = nx * ny;
    oz[0] = zm * s;
    oz[1] = z * s;
    oz[2] = zp * s;
  }
  // The same with the lattice's faces: beyond a mirror or wall face the
  // stencils see the edge node itself, the image of the node across the plane
  // half a node out (zero normal gradient).
  __host__ __device__ __forceinline__ void init_faces(int x, int y, int z, int nx, int ny,
                                                      int nz, const int (&face)[6]) {
    init(x, y, z, nx, ny, nz);
    if (x == 0 && face[0]) ox[0] = 0;
    if (x + 1 == nx && face[1]) ox[2] = nx - 1;
    if (y == 0 && face[2]) oy[0] = 0;
    if (y + 1 == ny && face[3]) oy[2] = (ny - 1) * nx;
    if (z == 0 && face[4]) oz[0] = 0;
    if (z + 1 == nz && face[5]) oz[2] = (nz - 1) * nx * ny;
  }
  template <class L>
  __host__ __device__ __forceinline__ int plus(int i) const {  // x + c_i
    return g(ox[L::cx(i) + 1] + oy[L::cy(i) + 1] + oz[L::cz(i) + 1]);
  }
  template <class L>
  __host__ __device__ __forceinline__ int minus(int i) const {  // x - c_i
    return g(ox[1 - L::cx(i)] + oy[1 - L::cy(i)] + oz[1 - L::cz(i)]);
  }
  // x + c_i for a direction known only at run time (selects without indexing
  // the offset arrays dynamically, so they stay in registers)
  template <class L>
  __host__ __device__ __forceinline__ int plus_rt(int i) const {
    const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
    return g((cx < 0 ? ox[0] : cx > 0 ? ox[2] : ox[1]) + (cy < 0 ? oy[0] : cy > 0 ? oy[2] : oy[1]) +
             (cz < 0 ? oz[0] : cz > 0 ? oz[2] : oz[1]));
  }
};

// Streaming across the lattice's faces, for the population pulled into
// direction j at node (x, y, z).  Returns 0 when x - c_j lies inside (or across
// a periodic face); 2 across a wall face: halfway bounce-back, direction
// opp(j) read at the node itself; 1 across mirror faces only: specular
// reflection, the direction with its components normal to the crossed faces
// reversed, read at the image node (Hood::init_faces' x - c_j).  *k is the
// direction to read.
template <class L>
__device__ __forceinline__ int face_cross(const int (&face)[6], int x, int y, int z, int nx,
                                          int ny, int nz, int j, int *k) {
  const int cx = L::cx(j), cy = L::cy(j), cz = L::cz(j);
  const int tx = (cx > 0 && x == 0) ? face[0] : ((cx < 0 && x == nx - 1) ? face[1] : 0);
  const int ty = (cy > 0 && y == 0) ? face[2] : ((cy < 0 && y == ny - 1) ? face[3] : 0);
  const int tz = (cz > 0 && z == 0) ? face[4] : ((cz < 0 && z == nz - 1) ? face[5] : 0);
  *k = j;
  if (!(tx | ty | tz)) return 0;
  if (tx == 2 || ty == 2 || tz == 2) {
    *k = L::opp(j);
    return 2;
  }
  *k = lat_index<L>(tx ? -cx : cx, ty ? -cy : cy, tz ? -cz : cz);
  return 1;
}

// Node on a face that is not periodic.
__device__ __forceinline__ bool on_wall_face(const int (&face)[6], int x, int y, int z, int nx,
                                             int ny, int nz) {
  return (face[0] && (x == 0 || x == nx - 1)) || (face[2] && (y == 0 || y == ny - 1)) ||
         (face[4] && (z == 0 || z == nz - 1));
}

template <class T, class S>
__device__ __forceinline__ T load_f(const S *base, int off, int i, double w) {
  if constexpr (Store<S>::k16) return T(w) + T(Store<S>::dec(base[off]));
  else return T(Store<S>::dec(__ldg(base + off)));
}
template <class T, class S>
__device__ __forceinline__ T load_g(const S *base, int off) {
  if constexpr (Store<S>::k16) return T(Store<S>::dec(base[off]));
  else return T(__ldg(base + off));
}

// Link fraction of the interpolated bounce-back (Sec. II.B, Eq. [eqn:tanh] and
// D = |x / (n.d)|): the fluid node sits x_s = 2 alpha_s artanh(2 C1 - 1) <= 0
// from the C1 = 1/2 surface; along link i the wall is q |c_i| away with
// q = |x_s / (n.d)| / |c_i|, n = G[C1]/|G[C1]|, d = c_i/|c_i|.  C1 is clamped to
// [1e-9, 1/2]; a degenerate normal, a link not pointing into the solid or
// q > 1 gives q = 1/2 (halfway bounce-back).
template <class L, class T>
__device__ __forceinline__ T link_q(T c1x, const T (&gc1)[3], int i, T alpha_s) {
  T c = c1x < T(1e-9) ? T(1e-9) : (c1x > T(0.5) ? T(0.5) : c1x);
  T xs = T(2) * alpha_s * atanh(T(2) * c - T(1));
  T gn = sqrt(gc1[0] * gc1[0] + gc1[1] * gc1[1] + gc1[2] * gc1[2]);
  if (!(gn >= T(1e-12))) return T(0.5);
  const int l2 = L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
  T cl = l2 == 1 ? T(1) : sqrt(T(l2));
  T nd = (gc1[0] * T(L::cx(i)) + gc1[1] * T(L::cy(i)) + gc1[2] * T(L::cz(i))) / (gn * cl);
  if (!(nd > T(1e-6))) return T(0.5);
  T q = fabs(xs / nd) / cl;
  return q > T(1) ? T(0.5) : q;
}

// The same link fraction from the node's precomputed x_s and |G[C1]|.
// link_fraction_rt: for a direction known only at run time (a rolled wall-link
// loop); link_fraction: for a direction known at compile time (an unrolled
// loop: the length of c_i and its components are constants).  The same
// arithmetic in the same order.
template <class L, class T>
__device__ __noinline__ T link_fraction_rt(T xs, T gn, T g0, T g1, T g2, int i) {
  if (!(gn >= T(1e-12))) return T(0.5);
  const int l2 = L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
  const T cl = l2 == 1 ? T(1) : sqrt(T(l2));
  const T nd = (g0 * T(L::cx(i)) + g1 * T(L::cy(i)) + g2 * T(L::cz(i))) / (gn * cl);
  if (!(nd > T(1e-6))) return T(0.5);
  const T q = fabs(xs / nd) / cl;
  return q > T(1) ? T(0.5) : q;
}
template <class L, class T>
__device__ __forceinline__ T link_fraction(T xs, T gn, T g0, T g1, T g2, int i) {
  if (!(gn >= T(1e-12))) return T(0.5);
  const int l2 = L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
  const T cl = l2 == 1 ? T(1) : sqrt(T(l2));
  const T nd = (g0 * T(L::cx(i)) + g1 * T(L::cy(i)) + g2 * T(L::cz(i))) / (gn * cl);
  if (!(nd > T(1e-6))) return T(0.5);
  const T q = fabs(xs / nd) / cl;
  return q > T(1) ? T(0.5) : q;
}

// ---------------------------------------------------------------------------
// K1: moments pass.  C(x) = sum_i g_i after streaming (Sec. II.B, C = sum g).
// FC: the lattice has a mirror or wall face; without one the face code is
// compiled out (here and in the fused pass), so periodic lattices keep their
// register count.
// ---------------------------------------------------------------------------
template <int K, class T, class S, bool FC>
__device__ __forceinline__ void moments_body(const LBArgs<T, S> &a, int x, int y, int z) {
  using L = Lat<K>;
  if (x >= a.nx || y >= a.ny || z >= a.nz) return;
  Hood h;
  if constexpr (FC) h.init_faces(x, y, z, a.nx, a.ny, a.nz, a.p.face);
  else h.init(x, y, z, a.nx, a.ny, a.nz);
  h.guard(a.err);
  const int n = h.g(h.ox[1] + h.oy[1] + h.oz[1]);
  // the moving populations are small next to the rest one (g_0 ~ C): summing
  // them first and adding g_0 last rounds once at the scale of C instead of
  // Q - 1 times, which keeps FP32 from drifting the liquid mass
  const T g0 = Store<S>::k16 ? T(a.g0_in[n]) : load_g<T, S>(a.gin[0], n);
  T s = T(0);
  if (FC && on_wall_face(a.p.face, x, y, z, a.nx, a.ny, a.nz)) {
    // a node on a mirror or wall face: the pulled g follow the face rules
#pragma unroll
    for (int i = 1; i < L::Q; i++) {
      int k;
      const int cr = face_cross<L>(a.p.face, x, y, z, a.nx, a.ny, a.nz, i, &k);
      const int src = cr == 2 ? n : h.plus_rt<L>(L::opp(i));
      s += load_g<T, S>(a.gin[k], src);
    }
    a.C[n] = g0 + s;
    return;
  }
#pragma unroll
  for (int i = 1; i < L::Q; i++) s += load_g<T, S>(a.gin[i], h.minus<L>(i));
  a.C[n] = g0 + s;
}

template <int K, class T, class S, bool FC>
__global__ void __launch_bounds__(256) moments_kernel(LBArgs<T, S> a) {
  moments_body<K, T, S, FC>(a, blockIdx.x * blockDim.x + threadIdx.x,
                        blockIdx.y * blockDim.y + threadIdx.y, blockIdx.z * blockDim.z + threadIdx.z);
}

// c_i . u for a direction known at compile time (adds only the non-zero
// components, in x, y, z order)
template <class L, class T>
__device__ __forceinline__ T cdot(int i, T ux, T uy, T uz) {
  T s = L::cx(i) == 0 ? T(0) : (L::cx(i) > 0 ? ux : -ux);
  if (L::cy(i)) s += L::cy(i) > 0 ? uy : -uy;
  if (L::cz(i)) s += L::cz(i) > 0 ? uz : -uz;
  return s;
}

// g_eq_i / w_i for i != 0 from a node's A = mu - 3/2 C u.u, C and cu = c_i.u:
//   mu + C s_i = A + C cu (3 + 9/2 cu)        (s_i of Eq. [eqn:feq], c_s^2 = 1/3)
template <class T>
__device__ __forceinline__ T geq_core(T A, T C, T cu) {
  return A + C * (cu * (T(3) + T(4.5) * cu));
}

// K1 with g held as g_eq: C(x) = sum_i g_eq_i(x - c_i), written as the node's
// own C plus the net inflow, so that the O(1) value is rounded once:
//   C(x) + [ sum_{i != 0} w_i (A + C cu (3 + 9/2 cu))(x - c_i)
//            - (1 - w_0) A(x) - 3/2 C(x) u(x).u(x) ]
// (sum_{i != 0} w_i c_i.u (3 + 9/2 c_i.u) = 3/2 u.u reduces the node's own
// outflow to its last two terms).  Ay, Cy, uy hold the values at x - c_i
// (index 0: the node itself).  Every moments pass of this form goes through
// this function, so that all of them round alike.
template <class L, class T>
__device__ __forceinline__ T moments_eq_node(const T (&Ay)[L::Q], const T (&Cy)[L::Q],
                                             const T (&uy)[L::Q][3]) {
  // axis and diagonal links (one weight each).  Link by link: pairing the
  // opposite links as the N-fluid rebuild does cost registers here (the
  // one-pass kernel spilled and ran 4 % slower).
  T sa = T(0), sd = T(0);
#pragma unroll
  for (int i = 1; i < L::Q; i++) {
    const T v = geq_core(Ay[i], Cy[i], cdot<L>(i, uy[i][0], uy[i][1], uy[i][2]));
    if (L::w(i) == L::w(1)) sa += v;
    else sd += v;
  }
  const T uu0 = uy[0][0] * uy[0][0] + uy[0][1] * uy[0][1] + uy[0][2] * uy[0][2];
  const T out = T(1.0 - L::w(0)) * Ay[0] + T(1.5) * Cy[0] * uu0;
  return Cy[0] + ((T(L::w(1)) * sa + T(L::w(L::Q - 1)) * sd) - out);
}

template <int K, class T, class S>
__device__ __forceinline__ void moments_eq_body(const LBArgs<T, S> &a, int x, int y, int z) {
  using L = Lat<K>;
  constexpr int Q = L::Q;
  if (x >= a.nx || y >= a.ny || z >= a.nz) return;
  Hood h;
  h.init(x, y, z, a.nx, a.ny, a.nz);
  h.guard(a.err);
  const int n = h.g(h.ox[1] + h.oy[1] + h.oz[1]);
  const T *pA = a.Mp[0], *pux = a.Mp[1], *puy = a.Mp[2], *puz = a.Mp[3];
  T Ay[Q], Cy[Q], uy[Q][3];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const int m = i == 0 ? n : h.minus<L>(i);
    Ay[i] = __ldg(pA + m);
    Cy[i] = __ldg(a.Cprev + m);
    uy[i][0] = (i == 0 || L::cx(i)) ? __ldg(pux + m) : T(0);
    uy[i][1] = (i == 0 || L::cy(i)) ? __ldg(puy + m) : T(0);
    uy[i][2] = (L::D == 3 && (i == 0 || L::cz(i))) ? __ldg(puz + m) : T(0);
  }
  a.C[n] = moments_eq_node<L, T>(Ay, Cy, uy);
}

// The same pass for D3Q19, tiled: a 32 x 4 block walks a run of zrun z planes.
// Each plane of (A, C, u) over the tile and a one-node halo is copied once into
// a five-plane shared ring by asynchronous copies (cp.async), three planes
// ahead of the plane being summed, and the five in-plane "cross" points (0,0),
// (+-1,0), (0,+-1) a node needs from planes z-1, z, z+1 stay in registers from
// one z to the next: per node 37 shared reads instead of 71 scattered loads.
// One barrier per plane.
constexpr int MT_X = 32, MT_Y = 4, MT_HX = MT_X + 2, MT_HY = MT_Y + 2, MT_RING = 5;

template <class T>
struct EqPt {
  T A, C, ux, uy, uz;
};
template <class T>
struct EqCross {
  EqPt<T> c, xm, xp, ym, yp;  // (0,0), (-1,0), (+1,0), (0,-1), (0,+1)
};

template <class T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <class T, class S>
__global__ void __launch_bounds__(MT_X * MT_Y, sizeof(T) == 8 ? 1 : 6)
    moments_eq_tiled_kernel(LBArgs<T, S> a, int zrun) {
  using L = Lat<1>;
  constexpr int NH = MT_HX * MT_HY;          // nodes of one staged plane
  constexpr int PER = (NH + MT_X * MT_Y - 1) / (MT_X * MT_Y);
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T(*sm)[MT_RING][NH] = reinterpret_cast<T(*)[MT_RING][NH]>(sm_raw);  // [field][slot][node]
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + MT_X * ty;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int x0 = blockIdx.x * MT_X, y0 = blockIdx.y * MT_Y;
  const int z0 = blockIdx.z * zrun, z1 = min(z0 + zrun, nz);
  const T *src[5] = {a.Mp[0], a.Cprev, a.Mp[1], a.Mp[2], a.Mp[3]};  // A, C, ux, uy, uz
  auto wrap = [](int v, int n) { v %= n; return v < 0 ? v + n : v; };
  // in-plane global index of the staged nodes this thread copies (-1: none)
  int hrow[PER];
#pragma unroll
  for (int r = 0; r < PER; r++) {
    const int k = tid + r * MT_X * MT_Y;
    hrow[r] = k < NH ? wrap(x0 - 1 + k % MT_HX, nx) + nx * wrap(y0 - 1 + k / MT_HX, ny) : -1;
  }
  auto issue = [&](int zz) {  // plane zz -> ring slot zz mod MT_RING, one copy group
    const int slot = wrap(zz, MT_RING);
    const long long zo = (long long)wrap(zz, nz) * nx * ny;
#pragma unroll
    for (int r = 0; r < PER; r++)
      if (hrow[r] >= 0) {
        const int k = tid + r * MT_X * MT_Y;
#pragma unroll
        for (int f = 0; f < 5; f++) cp_async_elem(&sm[f][slot][k], src[f] + zo + hrow[r]);
      }
    cp_async_commit();
  };
  auto pt = [&](int zz, int dx, int dy) {
    const int slot = wrap(zz, MT_RING);
    const int k = (tx + 1 + dx) + MT_HX * (ty + 1 + dy);
    EqPt<T> p;
    p.A = sm[0][slot][k];
    p.C = sm[1][slot][k];
    p.ux = sm[2][slot][k];
    p.uy = sm[3][slot][k];
    p.uz = sm[4][slot][k];
    return p;
  };
  auto cross = [&](int zz) {
    EqCross<T> c;
    c.c = pt(zz, 0, 0);
    c.xm = pt(zz, -1, 0);
    c.xp = pt(zz, 1, 0);
    c.ym = pt(zz, 0, -1);
    c.yp = pt(zz, 0, 1);
    return c;
  };
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < nx && y < ny;
  // one plane: wait for plane z + 1, refill the ring with plane z + 4 (into the
  // slot of plane z - 1, read for the last time in the previous step), then the
  // node's sum from the cross points of z - 1, z, z + 1 and the diagonals of z
  auto step = [&](int z, const EqCross<T> &Pm, const EqCross<T> &P0, EqCross<T> &Pp) {
    cp_async_wait<2>();  // planes up to z + 1 have landed (z + 2, z + 3 may be in flight)
    __syncthreads();
    issue(z + 4);
    Pp = cross(z + 1);
    if (active) {
      T Ay[L::Q], Cy[L::Q], uy[L::Q][3];
#pragma unroll
      for (int i = 0; i < L::Q; i++) {
        // the value at x - c_i: plane by -c_z, in-plane point by (-c_x, -c_y)
        const int sx = -L::cx(i), sy = -L::cy(i), sz = -L::cz(i);
        const EqCross<T> &Pl = sz < 0 ? Pm : (sz > 0 ? Pp : P0);
        EqPt<T> v;
        if (sx != 0 && sy != 0) v = pt(z, sx, sy);  // in-plane diagonal
        else v = sx < 0 ? Pl.xm : sx > 0 ? Pl.xp : sy < 0 ? Pl.ym : sy > 0 ? Pl.yp : Pl.c;
        Ay[i] = v.A;
        Cy[i] = v.C;
        uy[i][0] = (i == 0 || L::cx(i)) ? v.ux : T(0);
        uy[i][1] = (i == 0 || L::cy(i)) ? v.uy : T(0);
        uy[i][2] = (i == 0 || L::cz(i)) ? v.uz : T(0);
      }
      a.C[(long long)z * nx * ny + x + (long long)nx * y] = moments_eq_node<L, T>(Ay, Cy, uy);
    }
  };
  // prologue: planes z0 - 1 .. z0 + 3 in flight, the cross points of z0 - 1 and z0
  for (int d = -1; d <= 3; d++) issue(z0 + d);
  cp_async_wait<3>();
  __syncthreads();
  EqCross<T> Pa = cross(z0 - 1), Pb = cross(z0), Pc;
  // unrolled by three so that the rotating cross points stay in registers
  for (int z = z0; z < z1; z += 3) {
    step(z, Pa, Pb, Pc);
    if (z + 1 < z1) step(z + 1, Pb, Pc, Pa);
    if (z + 2 < z1) step(z + 2, Pc, Pa, Pb);
  }
  cp_async_wait<0>();  // no copy outlives the block
}

template <int K, class T, class S>
__global__ void __launch_bounds__(256) moments_eq_kernel(LBArgs<T, S> a) {
  moments_eq_body<K, T, S>(a, blockIdx.x * blockDim.x + threadIdx.x,
                           blockIdx.y * blockDim.y + threadIdx.y, blockIdx.z * blockDim.z + threadIdx.z);
}

// Where the fused pass finds C and C1 on the node's 1-neighbourhood, and where
// a collision of the g_eq form stores what fixes g (A = mu - 3/2 C u.u, u):
// global memory, as the per-lattice and batched launches keep them.  The
// single-pass step (dsm_zstep.cuh) reads both from shared memory instead.
struct GlobalIO {
  // wall links fixed in one rolled loop (fewer registers next to the
  // neighbourhood loads in flight); the f pulls of a solid node are issued
  // with the rest, before its C1 is known
  static constexpr bool kUnrollWall = false;
  static constexpr bool kSolidFirst = false;
  template <class L, class T, class S>
  __device__ __forceinline__ T C(const LBArgs<T, S> &a, const Hood &h, int i) const {
    return __ldg(a.C + h.plus<L>(i));
  }
  template <class L, class T, class S>
  __device__ __forceinline__ T C1(const LBArgs<T, S> &a, const Hood &h, int i) const {
    return __ldg(a.C1 + h.plus<L>(i));
  }
  // (C of this collision is the moments pass's output already in a.C)
  template <class L, class T, class S>
  __device__ __forceinline__ void put_eq(const LBArgs<T, S> &a, int n, T, T A, T ux, T uy,
                                         T uz) const {
    a.Mp[0][n] = A;
    a.Mp[1][n] = ux;
    a.Mp[2][n] = uy;
    if (L::D == 3) a.Mp[3][n] = uz;
  }
};

// ---------------------------------------------------------------------------
// K2: fused pass.  STAGE 2: fluids on the frozen diffuse solid C1.
// STAGE 1: relaxation of C1 itself (g carries C1; rho = 1, tau = tau_g = 1,
// every node fluid).  MODE_STEP collides and writes the next state;
// MODE_FIELDS writes one macroscopic field; MODE_OBS reduces observables.
// ---------------------------------------------------------------------------
template <int K, class T, class S, int STAGE, int MODE, bool RC, bool EQ, bool FC,
          class IO = GlobalIO>
__device__ __forceinline__ void node_body(const LBArgs<T, S> &a, int x, int y, int z, bool valid,
                                          int field_sel, const IO &io = IO()) {
  using L = Lat<K>;
  constexpr int Q = L::Q;
  // the pulled g enter only the g collision (C comes from the moments pass)
  constexpr bool LOAD_G = MODE == MODE_STEP && !EQ;
  static_assert(!EQ || STAGE == 2, "g as g_eq is a stage-2 form");
  static_assert(!(EQ && FC), "g as g_eq implies periodic faces");
  if (MODE != MODE_OBS && !valid) return;
  if (!valid) x = y = z = 0;
  Hood h;
  if constexpr (FC) h.init_faces(x, y, z, a.nx, a.ny, a.nz, a.p.face);
  else h.init(x, y, z, a.nx, a.ny, a.nz);
  h.guard(a.err);
  const int n = h.g(h.ox[1] + h.oy[1] + h.oz[1]);
  const ConstT<T> &K_ = a.c;

  // ---- every load of the node, issued up front ------------------------------
  // The populations are pulled from x - c_j for all j without a branch (a link
  // whose upstream node is solid is corrected below), so the 2Q population
  // loads and the 2Q neighbourhood loads are all in flight together.
  T C, c1, mu, rho, tau, omf, omg;  // omf = 1/tau, omg = 1/tau_g
  T gC[3] = {T(0), T(0), T(0)}, gR[3] = {T(0), T(0), T(0)}, gc1[3] = {T(0), T(0), T(0)};
  unsigned nb_solid = 0;  // bit k: x + c_k is solid (stage 2, fluid nodes next to the solid)
  T f[Q], g[Q];
  {
    T Cn[Q], C1n[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
      Cn[i] = io.template C<L>(a, h, i);
      C1n[i] = (STAGE == 2) ? io.template C1<L>(a, h, i) : T(0);
    }
#pragma unroll
    for (int j = 0; j < Q; j++) {
      const int src = h.minus<L>(j);
      if (!LOAD_G) g[j] = T(0);
      else if (Store<S>::k16 && j == 0) g[j] = T(a.g0_in[n]);
      else g[j] = load_g<T, S>(a.gin[j], src);
      if constexpr (IO::kSolidFirst) f[j] = T(L::w(j));
      else f[j] = load_f<T, S>(a.fin[j], src, j, L::w(j));
    }
    // the pulled f of a solid node (C1 >= 1/2) are never used: its collision
    // writes f* = w.  Where C1 of the node is at hand first (shared memory),
    // a solid node skips the pulls, and a warp of solid nodes issues none.
    if constexpr (IO::kSolidFirst) {
      if (!(STAGE == 2 && C1n[0] >= T(0.5))) {
#pragma unroll
        for (int j = 0; j < Q; j++) f[j] = load_f<T, S>(a.fin[j], h.minus<L>(j), j, L::w(j));
      }
    }
    C = Cn[0];
    c1 = C1n[0];
    T lapC = T(0), lapS = T(0);
    // the two Laplacian sums as one pair per neighbour (stage 2)
    Pr<T> lap2 = pr(T(0), T(0));
    const Pr<T> mc = pr(-C, -c1);
#pragma unroll
    for (int i = 1; i < Q; i++) {
      const T w = T(L::w(i));
      if (STAGE == 2) {
        lap2 = pr_fma(pr(w, w), pr_add(pr(Cn[i], C1n[i]), mc), lap2);
      } else {
        lapC += w * (Cn[i] - C);
      }
      if (L::cx(i)) gC[0] += w * T(L::cx(i)) * Cn[i];
      if (L::cy(i)) gC[1] += w * T(L::cy(i)) * Cn[i];
      if (L::cz(i)) gC[2] += w * T(L::cz(i)) * Cn[i];
    }
    if (STAGE == 2) {
      lapC = lap2.a;
      lapS = lap2.b;
    }
    lapC *= T(6);  // 2 / c_s^2
    lapS = lapC + T(6) * lapS;  // L[C1 + C] = L[C] + L[C1]
#pragma unroll
    for (int d = 0; d < 3; d++) gC[d] *= T(3);  // 1 / c_s^2
    if (STAGE == 2) {
      // Chemical potential of the frozen-solid free energy (Sec. II.B,
      // Eq. [eqn:fefrozen]), taken as its exact derivative in C2:
      //   mu = k2 b(C) + k3 b(C1 + C) - a^2 k2 L[C] - a^2 k3 L[C1 + C]
      mu = K_.k2 * bwell(C) + K_.k3 * bwell(c1 + C) - K_.a2k2 * lapC - K_.a2k3 * lapS;
      // density map rho = rho3 + (rho2 - rho3) C2/(C2 + C3), the ratio clamped
      // to [0, 1] and 0 where C2 + C3 = 1 - C1 <= 1e-6 (inside the solid)
      // (FP32: the volume fraction, clamped to [0, 1] right after, needs no
      // correctly rounded quotient -- the fast reciprocal-and-multiply division,
      // within 2 ulp, replaces a full IEEE division at every neighbour)
      auto rho_of = [&](T cc, T s1) -> T {
        const T den = T(1) - s1;
        T ph = T(0);
        if (den > T(1e-6)) {
          if constexpr (sizeof(T) == 4) ph = __fdividef(cc, den);
          else ph = cc / den;
          ph = ph < T(0) ? T(0) : (ph > T(1) ? T(1) : ph);
        }
        return K_.rho3 + K_.drho * ph;
      };
      rho = RC ? rho_of(C, c1) : K_.rho3;
      if (RC) {
#pragma unroll
        for (int i = 1; i < Q; i++) {
          const T r = T(L::w(i)) * rho_of(Cn[i], C1n[i]);
          if (L::cx(i)) gR[0] += r * T(L::cx(i));
          if (L::cy(i)) gR[1] += r * T(L::cy(i));
          if (L::cz(i)) gR[2] += r * T(L::cz(i));
        }
#pragma unroll
        for (int d = 0; d < 3; d++) gR[d] *= T(3);
      }
      // relaxation time map tau = tau3 + (tau2 - tau3) H(C2 - C3), H(0) = 0
      const bool liquid = C - (T(1) - c1 - C) > T(0);
      tau = liquid ? K_.tau2 : K_.tau3;
      omf = liquid ? K_.om2 : K_.om3;
      omg = K_.omg;
      // solid links (bit k: x + c_k is solid) only for a fluid node with a solid
      // neighbour -- rare; elsewhere one running max of C1 settles it
      T c1max = C1n[1];
#pragma unroll
      for (int i = 2; i < Q; i++) c1max = c1max > C1n[i] ? c1max : C1n[i];
      if (c1max >= T(0.5) && !(c1 >= T(0.5))) {
#pragma unroll
        for (int i = 1; i < Q; i++) nb_solid |= (C1n[i] >= T(0.5) ? 1u : 0u) << i;
#pragma unroll
        for (int i = 1; i < Q; i++) {
          const T w = T(L::w(i));
          if (L::cx(i)) gc1[0] += w * T(L::cx(i)) * C1n[i];
          if (L::cy(i)) gc1[1] += w * T(L::cy(i)) * C1n[i];
          if (L::cz(i)) gc1[2] += w * T(L::cz(i)) * C1n[i];
        }
#pragma unroll
        for (int d = 0; d < 3; d++) gc1[d] *= T(3);
      }
    } else {
      // Solid relaxation (Sec. II.B, Eq. [Free Energy1] and its chemical
      // potential): mu1 = (k1+k3) b(C1) - a^2 (k1+k3) L[C1]
      //   + 2 beta (C1 - 1/2) chi + 2 Omega C1 H(-C1) - 2 Omega (1 - C1) H(C1 - 1)
      // chi = 1 where the solid leaks out of S or the fluid into it (the
      // printed case labels of Eq. [frozen:poly-quadratic_lbm] read swapped).
      mu = K_.k13 * bwell(C) - K_.a2k13 * lapC;
      const bool inS = a.mask[n] != 0;
      if ((inS && C < T(0.5)) || (!inS && C > T(0.5))) mu += K_.beta2 * (C - T(0.5));
      if (C < T(0)) mu += K_.omega2 * C;
      if (C > T(1)) mu -= K_.omega2 * (T(1) - C);
      rho = T(1);
      tau = T(1);
      omf = T(1);
      omg = T(1);
    }
  }
  const bool solid_x = (STAGE == 2) && c1 >= T(0.5);

  // ---- interpolated bounce-back at the diffuse solid ------------------------
  // (only fluid nodes with a solid neighbour) -- replaces the pulled value of
  // every link whose upstream node x - c_j is solid.  Two forms of the same
  // arithmetic: one rolled loop over the directions, whose result goes to f[j]
  // through a select over all directions (IO::kUnrollWall false: the fewest
  // registers next to the neighbourhood loads of the global-memory pass), or
  // unrolled, so that a warp executes the body of a direction only when one of
  // its nodes has that wall link and each result lands in a fixed register.
  if (STAGE == 2 && !solid_x && (nb_solid & ~1u)) {
    // the node's distance to the C1 = 1/2 surface and the normal, once per node
    const T cc = c1 < T(1e-9) ? T(1e-9) : (c1 > T(0.5) ? T(0.5) : c1);
    const T xs = T(2) * K_.alpha_s * atanh(T(2) * cc - T(1));
    const T gn = sqrt(gc1[0] * gc1[0] + gc1[1] * gc1[1] + gc1[2] * gc1[2]);
    if constexpr (IO::kUnrollWall) {
#pragma unroll
      for (int j = 1; j < Q; j++) {
        const int i = L::opp(j);  // link from x toward the wall node x + c_i = x - c_j
        if ((nb_solid >> i) & 1u) {
          const T q = link_fraction<L, T>(xs, gn, gc1[0], gc1[1], gc1[2], i);
          const T fi_x = load_f<T, S>(a.fin[i], n, i, L::w(i));
          // x - c_i, the next fluid node away from the wall: with mirror or
          // wall faces it is pulled like any population (none beyond a wall)
          bool second = !((nb_solid >> j) & 1u);
          int ki = i;
          if constexpr (FC) {
            if (face_cross<L>(a.p.face, x, y, z, a.nx, a.ny, a.nz, i, &ki) == 2) second = false;
          }
          T v;
          if (q < T(0.5) && second) {
            const T fi_z = FC ? load_f<T, S>(a.fin[ki], h.plus<L>(j), ki, L::w(ki))
                              : load_f<T, S>(a.fin[i], h.plus<L>(j), i, L::w(i));
            v = T(2) * q * fi_x + (T(1) - T(2) * q) * fi_z;
          } else if (q < T(0.5)) {
            v = fi_x;  // no second fluid node: halfway rule
          } else {
            const T fj_x = load_f<T, S>(a.fin[j], n, j, L::w(j));
            v = (T(1) / (T(2) * q)) * fi_x + (T(1) - T(1) / (T(2) * q)) * fj_x;
          }
          f[j] = v;
        }
      }
    } else {
      for (int j = 1; j < Q; j++) {
        const int i = L::opp(j);  // link from x toward the wall node x + c_i = x - c_j
        if (!((nb_solid >> i) & 1u)) continue;
        const T q = link_fraction_rt<L, T>(xs, gn, gc1[0], gc1[1], gc1[2], i);
        const T fi_x = load_f<T, S>(a.fin[i], n, i, L::w(i));
        T v;
        int ki = i;
        bool second = !((nb_solid >> j) & 1u);
        if constexpr (FC) {
          if (face_cross<L>(a.p.face, x, y, z, a.nx, a.ny, a.nz, i, &ki) == 2) second = false;
        }
        if (q < T(0.5) && second) {
          const int z2 = h.plus_rt<L>(j);
          const T fi_z = load_f<T, S>(a.fin[ki], z2, ki, L::w(ki));
          v = T(2) * q * fi_x + (T(1) - T(2) * q) * fi_z;
        } else if (q < T(0.5)) {
          v = fi_x;  // no second fluid node: halfway rule
        } else {
          const T fj_x = load_f<T, S>(a.fin[j], n, j, L::w(j));
          v = (T(1) / (T(2) * q)) * fi_x + (T(1) - T(1) / (T(2) * q)) * fj_x;
        }
#pragma unroll
        for (int k = 1; k < Q; k++)
          if (k == j) f[k] = v;
      }
    }
  }

  // ---- mirror and wall faces -------------------------------------------------
  // Links across a face take its rule (specular reflection at a mirror,
  // halfway bounce-back at a wall) for f and g, except that a mirror link whose
  // image upstream node is solid keeps the interpolated value set above.
  // (unrolled over the directions, so that only a face node's crossing links do
  // work and every write is to a fixed register)
  if constexpr (FC) {
    if (on_wall_face(a.p.face, x, y, z, a.nx, a.ny, a.nz)) {
#pragma unroll
      for (int j = 1; j < Q; j++) {
        int k;
        const int cr = face_cross<L>(a.p.face, x, y, z, a.nx, a.ny, a.nz, j, &k);
        if (cr != 0) {
          const int src = cr == 2 ? n : h.plus_rt<L>(L::opp(j));
          const bool interp =
              STAGE == 2 && cr == 1 && !solid_x && ((nb_solid >> L::opp(j)) & 1u);
          if (!interp) f[j] = load_f<T, S>(a.fin[k], src, k, L::w(k));
          if (LOAD_G) g[j] = load_g<T, S>(a.gin[k], src);
        }
      }
    }
  }

  // ---- moments and forces --------------------------------------------------
  // Capillary force in its potential form mu G[C] (the form of the printed
  // velocity moment; it differs from -C G[mu] by the gradient G[C mu], a
  // pressure shift) plus the body force on the liquid, one total F in both the
  // forcing term and the velocity moment:
  //   rho u = sum_i c_i f_i + F/2,   pt = sum_i f_i + u.G[rho]/2  (pt = P/c_s^2)
  T u[3] = {T(0), T(0), T(0)}, pt = T(1), Fv[3];
  Fv[0] = mu * gC[0];
  Fv[1] = mu * gC[1];
  Fv[2] = mu * gC[2];
  if (STAGE == 2) {
    Fv[0] += C * K_.body[0];
    Fv[1] += C * K_.body[1];
    Fv[2] += C * K_.body[2];
  }
  if (!solid_x) {
    // opposite directions (j, j + 1) as one pair: their sum and difference in
    // one operation, the sum into the density, the difference into the
    // momentum (c_{j+1} = -c_j)
    T m0 = f[0], m1[3] = {T(0), T(0), T(0)};
    const Pr<T> pmj = pr(T(1), T(-1));
#pragma unroll
    for (int j = 1; j < Q; j += 2) {
      const Pr<T> sd = pr_fma(pr(f[j + 1], f[j + 1]), pmj, pr(f[j], f[j]));
      m0 += sd.a;
      if (L::cx(j)) m1[0] += T(L::cx(j)) * sd.b;
      if (L::cy(j)) m1[1] += T(L::cy(j)) * sd.b;
      if (L::cz(j)) m1[2] += T(L::cz(j)) * sd.b;
    }
    const T ir = (STAGE == 1) ? T(1) : (RC ? T(1) / rho : K_.inv_rho3);
    u[0] = (m1[0] + T(0.5) * Fv[0]) * ir;
    u[1] = (m1[1] + T(0.5) * Fv[1]) * ir;
    u[2] = (m1[2] + T(0.5) * Fv[2]) * ir;
    // (G[rho] = 0 without a density contrast)
    pt = RC ? m0 + T(0.5) * (u[0] * gR[0] + u[1] * gR[1] + u[2] * gR[2]) : m0;
  }
  const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];

  if constexpr (MODE == MODE_FIELDS) {
    T v;
    switch (field_sel) {
      case DSM_FIELD_C1: v = (STAGE == 2) ? c1 : C; break;
      case DSM_FIELD_C2: v = (STAGE == 2) ? C : T(0); break;
      case DSM_FIELD_C3: v = T(1) - ((STAGE == 2) ? c1 + C : C); break;
      case DSM_FIELD_MU: v = mu; break;
      case DSM_FIELD_UX: v = u[0]; break;
      case DSM_FIELD_UY: v = u[1]; break;
      case DSM_FIELD_UZ: v = u[2]; break;
      case DSM_FIELD_PT: v = pt; break;
      case DSM_FIELD_RHO: v = rho; break;
      default: v = tau; break;
    }
    a.fields[n] = v;
    return;
  }

  if constexpr (MODE == MODE_OBS) {
    bool bad = false;
#pragma unroll
    for (int j = 0; j < Q; j++) bad |= !solid_x && !isfinite(f[j]);
    bad |= !isfinite(C);  // C sums every pulled g
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    if constexpr (sizeof(T) == 4) {
      // FP32 lattices: carried-error sums in FP32 within a warp, FP64 beyond
      const float vals[OBS_K] = {valid ? float(C) : 0.f, valid ? float((STAGE == 2) ? c1 : C) : 0.f,
                                 valid ? 0.5f * float(rho) * float(uu) : 0.f,
                                 valid ? sqrtf(float(uu)) : 0.f, (valid && bad) ? 1.f : 0.f};
      const int is_max[OBS_K] = {0, 0, 0, 1, 1};
      block_reduce_ff<OBS_K>(vals, is_max, a.partials + b * OBS_K);
    } else {
      double vals[OBS_K];
      vals[0] = valid ? double(C) : 0.0;
      vals[1] = valid ? double((STAGE == 2) ? c1 : C) : 0.0;
      vals[2] = valid ? 0.5 * double(rho) * double(uu) : 0.0;
      vals[3] = valid ? sqrt(double(uu)) : 0.0;
      vals[4] = (valid && bad) ? 1.0 : 0.0;
      __shared__ double sh[OBS_K][32];
      const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
      const int lane = tid & 31, warp = tid >> 5;
      const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
#pragma unroll
      for (int k = 0; k < OBS_K; k++) {
        double v = vals[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double w2 = __shfl_down_sync(0xffffffffu, v, o);
          v = (k == 3 || k == 4) ? fmax(v, w2) : v + w2;
        }
        if (lane == 0) sh[k][warp] = v;
      }
      __syncthreads();
      if (tid < OBS_K) {
        double v = sh[tid][0];
        for (int w2 = 1; w2 < nw; w2++) v = (tid == 3 || tid == 4) ? fmax(v, sh[tid][w2]) : v + sh[tid][w2];
        a.partials[b * OBS_K + tid] = v;
      }
    }
    return;
  }

  // ---- BGK collision (Sec. II.B) -------------------------------------------
  //   s_i = c_i.u/c_s^2 + (c_i.u)^2/(2 c_s^4) - u.u/(2 c_s^2)
  //   f_eq_i = w_i (pt + rho s_i)                                 Eq. [eqn:feq]
  //   F_i = (1 - 1/(2 tau)) w_i [((c_i - u).G[rho]) s_i + c_i.F/c_s^2]
  //                                                       Eq. [eqn:hydroforce]
  //   g_eq_i = w_i (mu + C s_i) (i != 0),  g_eq_0 = C - (1 - w_0) mu + w_0 C s_0
  // (the minus signs read where the printed forms would break sum f_eq = pt and
  // sum g_eq = C).  Solid nodes: f* = w_i; g collides with u = 0.
  // Directions come in opposite pairs (i, i+1): c_{i+1} = -c_i, so s splits
  // into a shared even part and an odd part of opposite sign.  Without a density
  // contrast (RC = false) G[rho] = 0 and its forcing terms vanish exactly.
  if (!isfinite(pt + mu + u[0] + u[1] + u[2])) atomicOr(a.err, ERR_NONFINITE);
  const T kF = T(1) - T(0.5) * omf;
  const T kF3 = T(3) * kF;
  const T ug = RC ? u[0] * gR[0] + u[1] * gR[1] + u[2] * gR[2] : T(0);
  const T m15uu = T(1.5) * uu;
  T gsum16 = T(0);
  auto put_f = [&](int i, T fo) {
    if constexpr (Store<S>::k16) a.fout[i][n] = Store<S>::enc(float(fo - T(L::w(i))));
    else a.fout[i][n] = S(fo);
  };
  auto put_g = [&](int i, T go) {
    if constexpr (Store<S>::k16) {
      const S e = Store<S>::enc(float(go));
      a.gout[i][n] = e;
      gsum16 += T(Store<S>::dec(e));
    } else {
      a.gout[i][n] = S(go);
    }
  };
  {  // rest population
    const T w = T(L::w(0));
    const T s = -m15uu;
    T fo = w;
    if (!solid_x) {
      T Fi = T(0);
      if (RC) Fi = kF * w * (-ug * s);
      fo = f[0] + (w * (pt + rho * s) - f[0]) * omf + Fi;
    }
    put_f(0, fo);
    if constexpr (!EQ) {
      const T geq = C - (T(1) - w) * mu + w * C * s;
      const T go = g[0] + (geq - g[0]) * omg;
      if constexpr (!Store<S>::k16) a.gout[0][n] = S(go);
    }
  }
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int ib = i + 1;  // opposite direction
    const T w = T(L::w(i));
    const T cu = cdot<L>(i, u[0], u[1], u[2]);
    const T even = T(4.5) * cu * cu - m15uu;
    const T odd = T(3) * cu;
    // the opposite pair (i, ib) as one pair of values: s = even +- odd, and
    // every later operation once for both
    const Pr<T> pm = pr(T(1), T(-1)), m1 = pr(T(-1), T(-1));
    const Pr<T> s2 = pr_fma(pr(odd, odd), pm, pr(even, even));
    T fp = w, fm = w;
    if (!solid_x) {
      const T wpt = w * pt, wr = w * rho;
      const T cF = cdot<L>(i, Fv[0], Fv[1], Fv[2]);
      const T Fp = w * kF3 * cF;
      Pr<T> F2 = pr(Fp, -Fp);
      if (RC) {
        const T cg = cdot<L>(i, gR[0], gR[1], gR[2]);
        const T kw = kF * w;
        F2 = pr_fma(pr(kw, kw), pr_mul(pr(cg - ug, -cg - ug), s2), F2);
      }
      const Pr<T> f2 = pr(f[i], f[ib]);
      const Pr<T> eq = pr_fma(pr(wr, wr), s2, pr(wpt, wpt));  // w (pt + rho s)
      const Pr<T> o = pr_add(pr_fma(pr_fma(f2, m1, eq), pr(omf, omf), f2), F2);
      fp = o.a;
      fm = o.b;
    }
    put_f(i, fp);
    put_f(ib, fm);
    if constexpr (!EQ) {
      const T wmu = w * mu, wC = w * C;
      const Pr<T> g2 = pr(g[i], g[ib]);
      const Pr<T> geq = pr_fma(pr(wC, wC), s2, pr(wmu, wmu));
      const Pr<T> go = pr_fma(pr_fma(g2, m1, geq), pr(omg, omg), g2);
      put_g(i, go.a);
      put_g(ib, go.b);
    }
  }
  if constexpr (EQ) {
    // g* = g_eq (tau_g = 1): store what fixes it.  The C of this collision is
    // this step's moments output a.C, which the next step reads as Cprev.
    io.template put_eq<L>(a, n, C, mu - T(1.5) * C * uu, u[0], u[1], u[2]);
  } else if constexpr (Store<S>::k16) {
    // 16-bit storage: the rest population takes the rounding of the others so
    // that sum_i g*_i = C holds at every node (sum_i g_eq_i = C, so the exact
    // post-collision sum is C) and the liquid mass is conserved.
    a.g0_out[n] = float(C - gsum16);
  }
  (void)gsum16;
}

template <int K, class T, class S, int STAGE, int MODE, bool RC, bool EQ, bool FC>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : (EQ ? 3 : 2)) node_kernel(LBArgs<T, S> a, int field_sel) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  node_body<K, T, S, STAGE, MODE, RC, EQ, FC>(a, x, y, z, x < a.nx && y < a.ny && z < a.nz, field_sel);
}

// ---------------------------------------------------------------------------
// K9: batched persistent step.  One cooperative launch advances many lattices
// (same lattice kind and precision) by up to tmax steps: per step a moments
// phase and a fused phase over the work list of (lattice, brick) pairs, each
// phase followed by a grid-wide barrier.  Resident blocks walk the list in a
// grid-stride loop.  Every barrier wait is bounded: after `limit` polls
// (kBarrierSpins unless the caller set dsm_set_wait_limit) the block latches
// ERR_TIMEOUT in every lattice's error word and returns, so a lost block can
// never hang the GPU.  Per-node arithmetic is node_body /
// moments_body, the same code as the single-lattice step, so each lattice's
// result equals its solo result bitwise.
// ---------------------------------------------------------------------------
template <class T, class S>
struct BatchItem {
  LBArgs<T, S> a[2];  // a[p]: arguments while the lattice's current buffer is p
  int gx, gy, gz;     // bricks per axis
  int brick0;         // first brick of this lattice in the work list
  int nsteps;         // steps this launch takes for this lattice
  int cur0;           // current buffer at launch
  int implicit0;      // g held as g_eq at launch
};

constexpr unsigned long long kBarrierSpins = 20000000ull;  // ~2-4 s of polling

template <class T, class S>
__device__ bool grid_barrier(unsigned *bar, const BatchItem<T, S> *items, int nitems,
                             unsigned long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
    ok = 1;
    volatile unsigned *gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long spins = 0;
      while (*gen == g) {
        __nanosleep(100);
        if (++spins > limit) {
          for (int i = 0; i < nitems; i++) atomicOr(items[i].a[0].err, ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <int K, class T, class S, bool RC, bool EQ>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 2)
    batch_kernel(const BatchItem<T, S> *items, int nitems, const int *owner, int nbricks, int tmax,
                 unsigned *bar, unsigned long long spin_limit) {
  __shared__ LBArgs<T, S> sa;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  for (int t = 0; t < tmax; t++) {
    for (int phase = 0; phase < 2; phase++) {
      for (int b = blockIdx.x; b < nbricks; b += gridDim.x) {
        const BatchItem<T, S> *it = items + __ldg(owner + b);
        if (t >= it->nsteps) continue;  // uniform over the block
        __syncthreads();
        {  // this lattice's arguments for this step, into shared memory
          const int *src = (const int *)&it->a[(it->cur0 + t) & 1];
          int *dst = (int *)&sa;
          for (int w = tid; w < (int)(sizeof(LBArgs<T, S>) / sizeof(int)); w += nthr) dst[w] = src[w];
        }
        __syncthreads();
        const int lb = b - it->brick0;
        const int bx = lb % it->gx, by = (lb / it->gx) % it->gy, bz = lb / (it->gx * it->gy);
        const int x = bx * blockDim.x + threadIdx.x;
        const int y = by * blockDim.y + threadIdx.y;
        const int z = bz * blockDim.z + threadIdx.z;
        if (phase == 0) {
          if (EQ && (t > 0 || it->implicit0)) moments_eq_body<K, T, S>(sa, x, y, z);
          else moments_body<K, T, S, false>(sa, x, y, z);
        } else {
          node_body<K, T, S, 2, MODE_STEP, RC, EQ, false>(sa, x, y, z, x < sa.nx && y < sa.ny && z < sa.nz, 0);
        }
      }
      if (!grid_barrier<T, S>(bar, items, nitems, spin_limit)) return;
    }
  }
}

// ---------------------------------------------------------------------------
// K3: initial state at rest (reading of the unstated initial condition):
// f_i = w_i, g_i = g_eq_i(C, mu(C), u = 0), stored as the post-collision state.
// ---------------------------------------------------------------------------
template <int K, class T, class S, int STAGE>
__global__ void __launch_bounds__(256) init_kernel(LBArgs<T, S> a, const T *cfield) {
  using L = Lat<K>;
  constexpr int Q = L::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x >= a.nx || y >= a.ny || z >= a.nz) return;
  Hood h;
  h.init_faces(x, y, z, a.nx, a.ny, a.nz, a.p.face);
  h.guard(a.err);
  const int n = h.g(h.ox[1] + h.oy[1] + h.oz[1]);
  const ConstT<T> &K_ = a.c;
  const T C = cfield[n];
  const T c1 = (STAGE == 2) ? a.C1[n] : T(0);
  T lapC = T(0), lapS = T(0);
#pragma unroll
  for (int i = 1; i < Q; i++) {
    const int m = h.plus<L>(i);
    const T w = T(L::w(i));
    lapC += w * (cfield[m] - C);
    if (STAGE == 2) lapS += w * ((a.C1[m] + cfield[m]) - (c1 + C));
  }
  lapC *= T(6);
  lapS *= T(6);
  T mu;
  if (STAGE == 2) {
    mu = K_.k2 * bwell(C) + K_.k3 * bwell(c1 + C) - K_.a2k2 * lapC - K_.a2k3 * lapS;
  } else {
    mu = K_.k13 * bwell(C) - K_.a2k13 * lapC;
    const bool inS = a.mask[n] != 0;
    if ((inS && C < T(0.5)) || (!inS && C > T(0.5))) mu += K_.beta2 * (C - T(0.5));
    if (C < T(0)) mu += K_.omega2 * C;
    if (C > T(1)) mu -= K_.omega2 * (T(1) - C);
  }
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const T w = T(L::w(i));
    const long long off = (long long)i * a.pitch + n;
    if constexpr (Store<S>::k16) a.f_out[off] = Store<S>::enc(0.0f);
    else a.f_out[off] = S(w);
    const T geq = (i == 0) ? C - (T(1) - w) * mu : w * mu;
    if constexpr (Store<S>::k16) {
      if (i > 0) a.g_out[off] = Store<S>::enc(float(geq));
    } else {
      a.g_out[off] = S(geq);
    }
  }
  if constexpr (Store<S>::k16) {
    T s = T(0);
#pragma unroll
    for (int i = 1; i < Q; i++) s += T(Store<S>::dec(a.g_out[(long long)i * a.pitch + n]));
    a.g0_out[n] = float(C - s);
  }
}

// K7: analytic solid.  C1 = 1/2 + tanh(d / (2 alpha_s)) / 2 from the signed
// distance d (positive inside S): the planar profile of Sec. II.A,
// Eq. [frozen:interface_profile].
template <class T>
__global__ void __launch_bounds__(256) solid_profile_kernel(const T *sd, T *c1, long long N,
                                                            T alpha_s) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N;
       k += (long long)gridDim.x * blockDim.x)
    c1[k] = T(0.5) + T(0.5) * tanh(sd[k] / (T(2) * alpha_s));
}

// Population codecs (test/checkpoint path): storage <-> reals, q-major N-stride.
// With g held as g_eq (implicit), g is rebuilt from (A, u, Cprev) with the
// arithmetic of the moments pass: g_i = w_i (A + C c_i.u (3 + 9/2 c_i.u)),
// g_0 = C - (1 - w_0) A - 3/2 C u.u.
template <int K, class T, class S>
__global__ void __launch_bounds__(256) pops_get_kernel(LBArgs<T, S> a, T *fo, T *go, int implicit) {
  using L = Lat<K>;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < a.N;
       k += (long long)gridDim.x * blockDim.x) {
    T A = T(0), Cx = T(0), ux = T(0), uy = T(0), uz = T(0);
    if (implicit) {
      A = a.Mp[0][k];
      Cx = a.Cprev[k];
      ux = a.Mp[1][k];
      uy = a.Mp[2][k];
      uz = L::D == 3 ? a.Mp[3][k] : T(0);
    }
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
      const long long off = (long long)i * a.pitch + k;
      if constexpr (Store<S>::k16) fo[i * a.N + k] = T(L::w(i)) + T(Store<S>::dec(a.f_in[off]));
      else fo[i * a.N + k] = T(a.f_in[off]);
      if (implicit) {
        go[i * a.N + k] = i == 0 ? Cx - (T(1.0 - L::w(0)) * A + T(1.5) * Cx * (ux * ux + uy * uy + uz * uz))
                                 : T(L::w(i)) * geq_core(A, Cx, cdot<L>(i, ux, uy, uz));
      } else if constexpr (Store<S>::k16) {
        go[i * a.N + k] = (i == 0) ? T(a.g0_in[k]) : T(Store<S>::dec(a.g_in[off]));
      } else {
        go[i * a.N + k] = T(a.g_in[off]);
      }
    }
  }
}

// g held as g_eq -> stored populations of the current buffer (a.g_out), for a
// switch to the population form.  16-bit storage keeps the node's sum exact
// through g_0 as the fused pass does.
template <int K, class T, class S>
__global__ void __launch_bounds__(256) g_materialize_kernel(LBArgs<T, S> a) {
  using L = Lat<K>;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < a.N;
       k += (long long)gridDim.x * blockDim.x) {
    const T A = a.Mp[0][k], Cx = a.Cprev[k], ux = a.Mp[1][k], uy = a.Mp[2][k];
    const T uz = L::D == 3 ? a.Mp[3][k] : T(0);
    T s16 = T(0);
#pragma unroll
    for (int i = 1; i < L::Q; i++) {
      const T gi = T(L::w(i)) * geq_core(A, Cx, cdot<L>(i, ux, uy, uz));
      const long long off = (long long)i * a.pitch + k;
      if constexpr (Store<S>::k16) {
        a.g_out[off] = Store<S>::enc(float(gi));
        s16 += T(Store<S>::dec(a.g_out[off]));
      } else {
        a.g_out[off] = S(gi);
      }
    }
    if constexpr (Store<S>::k16) a.g0_out[k] = float(Cx - s16);
    else a.g_out[k] = S(Cx - (T(1.0 - L::w(0)) * A + T(1.5) * Cx * (ux * ux + uy * uy + uz * uz)));
  }
}

template <int K, class T, class S>
__global__ void __launch_bounds__(256) pops_set_kernel(LBArgs<T, S> a, const T *fi, const T *gi) {
  using L = Lat<K>;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < a.N;
       k += (long long)gridDim.x * blockDim.x) {
    T gs = T(0), g0 = T(0);
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
      const long long off = (long long)i * a.pitch + k;
      const T fv = fi[i * a.N + k], gv = gi[i * a.N + k];
      if constexpr (Store<S>::k16) {
        a.f_out[off] = Store<S>::enc(float(fv - T(L::w(i))));
        if (i == 0) {
          g0 = gv;
        } else {
          a.g_out[off] = Store<S>::enc(float(gv));
          gs += T(Store<S>::dec(a.g_out[off])) - gv;
        }
      } else {
        a.f_out[off] = S(fv);
        a.g_out[off] = S(gv);
      }
    }
    // 16-bit: keep the node's sum of g as given
    if constexpr (Store<S>::k16) a.g0_out[k] = float(g0 - gs);
  }
}

}  // namespace dsm

#include "dsm_zstep.cuh"

namespace dsm {

// ---------------------------------------------------------------------------
// Host side: typed launchers behind a type-erased table.
// ---------------------------------------------------------------------------
// Block shape of the per-lattice launches.  Lattices too small to give every SM
// a 256-thread block (fewer than ~2 x 152 x 256 nodes) use 64-thread blocks so
// that their work spreads over four times as many SMs.  Larger lattices: shapes
// measured on the fused pass (D3Q19 FP32, g held as g_eq), best kept --
//   256x256x192:  32x4x2 0.510 ms, 64x4x1 0.494, 128x2x1 0.486, 256x1x1 0.484;
//                 later, on the current kernel: 256x1x1 0.4742, 128x1x1 0.4678,
//                 64x1x1 0.4710 (128x1x1 also best for the population form and
//                 for D2Q9 at 4096^2);
//   384x384x256:  32x4x2 1.784 ms, 64x4x1 1.784, 64x2x2 1.772, 128x2x1 2.025,
//                 128x1x2 2.017.
//   384x384x256, later: 64x2x2 1.7357 ms, 128x1x1 1.7138.
// 128-node rows where nx is a multiple of 128, else 64x2x2, else 32-wide bricks.  The
// batched launch keeps 32-wide bricks for every lattice (lb_block_batch), which
// suits its small lattices.
inline dim3 lb_block_batch(int kind) { return kind == 0 ? dim3(32, 8, 1) : dim3(32, 4, 2); }
inline dim3 lb_block(int kind, int nx, int ny, int nz) {
  if ((long long)nx * ny * nz < 2ll * 152 * 256) return kind == 0 ? dim3(32, 2, 1) : dim3(32, 1, 2);
  if (nx % 128 == 0) return dim3(128, 1, 1);  // rows of 128: more, smaller blocks per SM
  if (nx % 64 == 0) return kind == 0 ? dim3(64, 4, 1) : dim3(64, 2, 2);
  return lb_block_batch(kind);
}
inline dim3 lb_grid_of(dim3 b, int nx, int ny, int nz) {
  return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y, (nz + b.z - 1) / b.z);
}
inline dim3 lb_grid(int kind, int nx, int ny, int nz) {
  const dim3 b = lb_block(kind, nx, ny, nz);
  return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y, (nz + b.z - 1) / b.z);
}

template <class T, class S>
LBArgs<T, S> typed(const LBRaw &r) {
  LBArgs<T, S> a;
  a.nx = r.nx; a.ny = r.ny; a.nz = r.nz; a.N = r.N; a.pitch = r.pitch;
  a.f_in = (const S *)r.f_in; a.g_in = (const S *)r.g_in; a.g0_in = r.g0_in;
  a.f_out = (S *)r.f_out; a.g_out = (S *)r.g_out; a.g0_out = r.g0_out;
  a.C = (T *)r.C; a.Cprev = (const T *)r.Cprev; a.C1 = (const T *)r.C1; a.mask = r.mask;
  for (int k = 0; k < 4; k++) a.Mp[k] = r.M ? (T *)r.M + (long long)k * r.pitch : nullptr;
  a.Qz = (T *)r.Qz;
  a.Uz = (T *)r.Uz;
  a.nxp = r.nxp;
  a.nyp = r.nyp;
  a.fields = (T *)r.out; a.partials = r.partials; a.err = r.err; a.p = r.p;
  a.c = ConstT<T>::make(r.p);
  for (int i = 0; i < QMAX; i++) {
    const long long o = (long long)i * r.pitch;
    a.fin[i] = a.f_in ? a.f_in + o : nullptr;
    a.gin[i] = a.g_in ? a.g_in + o : nullptr;
    a.fout[i] = a.f_out ? a.f_out + o : nullptr;
    a.gout[i] = a.g_out ? a.g_out + o : nullptr;
  }
  return a;
}

// The same pass for D2Q9, tiled: a 32 x 8 block (T2_X x T2_Y: 32 x 4 measured
// 10 % slower here) stages (A, C, u_x, u_y) of its
// tile and a one-node halo in shared memory once, then each node sums its nine
// points from there (the per-node arithmetic is moments_eq_node, as above).
constexpr int T2_X = 32, T2_Y = 8, T2_HX = T2_X + 2, T2_HY = T2_Y + 2;
template <class T, class S>
__global__ void __launch_bounds__(T2_X * T2_Y) moments_eq_tiled2d_kernel(LBArgs<T, S> a) {
  using L = Lat<0>;
  constexpr int NH = T2_HX * T2_HY;
  __shared__ T sA[NH], sC[NH], sU[NH], sV[NH];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + T2_X * ty;
  const int nx = a.nx, ny = a.ny;
  const int x0 = blockIdx.x * T2_X, y0 = blockIdx.y * T2_Y;
  auto wrap = [](int v, int n) { v %= n; return v < 0 ? v + n : v; };
  for (int k = tid; k < NH; k += T2_X * T2_Y) {
    const int g = wrap(x0 - 1 + k % T2_HX, nx) + nx * wrap(y0 - 1 + k / T2_HX, ny);
    sA[k] = __ldg(a.Mp[0] + g);
    sC[k] = __ldg(a.Cprev + g);
    sU[k] = __ldg(a.Mp[1] + g);
    sV[k] = __ldg(a.Mp[2] + g);
  }
  __syncthreads();
  const int x = x0 + tx, y = y0 + ty;
  if (x >= nx || y >= ny) return;
  T Ay[L::Q], Cy[L::Q], uy[L::Q][3];
#pragma unroll
  for (int i = 0; i < L::Q; i++) {
    const int k = (tx + 1 - L::cx(i)) + T2_HX * (ty + 1 - L::cy(i));  // x - c_i
    Ay[i] = sA[k];
    Cy[i] = sC[k];
    uy[i][0] = (i == 0 || L::cx(i)) ? sU[k] : T(0);
    uy[i][1] = (i == 0 || L::cy(i)) ? sV[k] : T(0);
    uy[i][2] = T(0);
  }
  a.C[x + (long long)nx * y] = moments_eq_node<L, T>(Ay, Cy, uy);
}

template <class T>
constexpr size_t moments_eq_smem() {
  return sizeof(T) * 5 * MT_RING * MT_HX * MT_HY;
}

template <int K, class T, class S>
struct LBOps {
  static cudaError_t moments(const LBRaw &r, cudaStream_t st) {
    const dim3 g = lb_grid(K, r.nx, r.ny, r.nz), b = lb_block(K, r.nx, r.ny, r.nz);
    if (r.implicit && K == 1 && moments_eq_smem<T>() > 48 * 1024) {
      static bool opted_in = false;  // above 48 KB of dynamic shared memory
      if (!opted_in) {
        const cudaError_t e = cudaFuncSetAttribute(moments_eq_tiled_kernel<T, S>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)moments_eq_smem<T>());
        if (e != cudaSuccess) return e;
        opted_in = true;
      }
    }
    if (r.implicit && K == 1) {
      // the longest run of z planes (fewer ring refills per plane) that still
      // fills one wave of six 128-thread blocks per SM
      const int tiles = ((r.nx + MT_X - 1) / MT_X) * ((r.ny + MT_Y - 1) / MT_Y);
      int zrun = 32;
      while (zrun > 4 && (long long)tiles * ((r.nz + zrun - 1) / zrun) < 6 * 152) zrun /= 2;
      moments_eq_tiled_kernel<T, S><<<dim3((r.nx + MT_X - 1) / MT_X, (r.ny + MT_Y - 1) / MT_Y,
                                           (r.nz + zrun - 1) / zrun),
                                      dim3(MT_X, MT_Y, 1), moments_eq_smem<T>(), st>>>(typed<T, S>(r), zrun);
    } else if (r.implicit && K == 0 && (long long)r.nx * r.ny >= 2ll * 152 * 256) {
      moments_eq_tiled2d_kernel<T, S><<<dim3((r.nx + T2_X - 1) / T2_X, (r.ny + T2_Y - 1) / T2_Y),
                                        dim3(T2_X, T2_Y, 1), 0, st>>>(typed<T, S>(r));
    } else if (r.implicit) moments_eq_kernel<K, T, S><<<g, b, 0, st>>>(typed<T, S>(r));
    else if (r.p.walls) moments_kernel<K, T, S, true><<<g, b, 0, st>>>(typed<T, S>(r));
    else moments_kernel<K, T, S, false><<<g, b, 0, st>>>(typed<T, S>(r));
    return cudaGetLastError();
  }
  template <int STAGE, int MODE, bool EQ, bool FC>
  static void node_launch_fc(const LBRaw &r, cudaStream_t st) {
    const dim3 g = lb_grid(K, r.nx, r.ny, r.nz), b = lb_block(K, r.nx, r.ny, r.nz);
    if (STAGE == 2 && r.p.rho_contrast)
      node_kernel<K, T, S, STAGE, MODE, STAGE == 2, EQ, FC><<<g, b, 0, st>>>(typed<T, S>(r), r.field_sel);
    else
      node_kernel<K, T, S, STAGE, MODE, false, EQ, FC><<<g, b, 0, st>>>(typed<T, S>(r), r.field_sel);
  }
  template <int STAGE, int MODE, bool EQ = false>
  static void node_launch(const LBRaw &r, cudaStream_t st) {
    // (g held as g_eq implies periodic faces)
    if (!EQ && r.p.walls) node_launch_fc<STAGE, MODE, false, true>(r, st);
    else node_launch_fc<STAGE, MODE, EQ, false>(r, st);
  }
  static cudaError_t node(const LBRaw &r, int stage, int mode, cudaStream_t st) {
    if (stage == 2) {
      if (mode == MODE_STEP && r.eq) node_launch<2, MODE_STEP, true>(r, st);
      else if (mode == MODE_STEP) node_launch<2, MODE_STEP>(r, st);
      else if (mode == MODE_FIELDS) node_launch<2, MODE_FIELDS>(r, st);
      else node_launch<2, MODE_OBS>(r, st);
    } else {
      if (mode == MODE_STEP) node_launch<1, MODE_STEP>(r, st);
      else if (mode == MODE_FIELDS) node_launch<1, MODE_FIELDS>(r, st);
      else node_launch<1, MODE_OBS>(r, st);
    }
    return cudaGetLastError();
  }
  static cudaError_t init(const LBRaw &r, const void *cfield, int stage, cudaStream_t st) {
    if (stage == 2)
      init_kernel<K, T, S, 2><<<lb_grid(K, r.nx, r.ny, r.nz), lb_block(K, r.nx, r.ny, r.nz), 0, st>>>(
          typed<T, S>(r), (const T *)cfield);
    else
      init_kernel<K, T, S, 1><<<lb_grid(K, r.nx, r.ny, r.nz), lb_block(K, r.nx, r.ny, r.nz), 0, st>>>(
          typed<T, S>(r), (const T *)cfield);
    return cudaGetLastError();
  }
  static cudaError_t solid(const void *sd, void *c1, long long N, double alpha_s, cudaStream_t st) {
    const int blocks = (int)((N + 255) / 256 < 152 * 32 ? (N + 255) / 256 : 152 * 32);
    solid_profile_kernel<T><<<blocks > 0 ? blocks : 1, 256, 0, st>>>((const T *)sd, (T *)c1, N,
                                                                     T(alpha_s));
    return cudaGetLastError();
  }
  static cudaError_t get_pops(const LBRaw &r, void *fo, void *go, cudaStream_t st) {
    const int blocks = (int)((r.N + 255) / 256 < 152 * 32 ? (r.N + 255) / 256 : 152 * 32);
    pops_get_kernel<K, T, S><<<blocks > 0 ? blocks : 1, 256, 0, st>>>(typed<T, S>(r), (T *)fo,
                                                                      (T *)go, r.implicit);
    return cudaGetLastError();
  }
  static cudaError_t materialize(const LBRaw &r, cudaStream_t st) {
    const int blocks = (int)((r.N + 255) / 256 < 152 * 32 ? (r.N + 255) / 256 : 152 * 32);
    g_materialize_kernel<K, T, S><<<blocks > 0 ? blocks : 1, 256, 0, st>>>(typed<T, S>(r));
    return cudaGetLastError();
  }
  static cudaError_t set_pops(const LBRaw &r, const void *fi, const void *gi, cudaStream_t st) {
    const int blocks = (int)((r.N + 255) / 256 < 152 * 32 ? (r.N + 255) / 256 : 152 * 32);
    pops_set_kernel<K, T, S><<<blocks > 0 ? blocks : 1, 256, 0, st>>>(typed<T, S>(r),
                                                                      (const T *)fi, (const T *)gi);
    return cudaGetLastError();
  }
  static size_t batch_bytes(const BatchRaw *items, int n) {
    long long bricks = 0;
    for (int i = 0; i < n; i++) {
      const dim3 g = lb_grid_of(lb_block_batch(K), items[i].r[0].nx, items[i].r[0].ny, items[i].r[0].nz);
      bricks += (long long)g.x * g.y * g.z;
    }
    return 256 + (size_t)round_up((long long)n * sizeof(BatchItem<T, S>), 256) +
           (size_t)round_up(bricks * (long long)sizeof(int), 256);
  }
  static cudaError_t batch(const BatchRaw *items, int n, void *scratch, size_t bytes, bool rc,
                           bool eq, unsigned long long spins, cudaStream_t st) {
    if (bytes < batch_bytes(items, n)) return cudaErrorInvalidValue;
    std::vector<BatchItem<T, S>> hi(n);
    std::vector<int> owner;
    int tmax = 0;
    for (int i = 0; i < n; i++) {
      BatchItem<T, S> &b = hi[i];
      b.a[0] = typed<T, S>(items[i].r[0]);
      b.a[1] = typed<T, S>(items[i].r[1]);
      const dim3 g = lb_grid_of(lb_block_batch(K), items[i].r[0].nx, items[i].r[0].ny, items[i].r[0].nz);
      b.gx = g.x;
      b.gy = g.y;
      b.gz = g.z;
      b.brick0 = (int)owner.size();
      b.nsteps = (int)items[i].nsteps;
      b.cur0 = items[i].cur0;
      b.implicit0 = items[i].r[0].implicit;
      if (b.nsteps > tmax) tmax = b.nsteps;
      owner.insert(owner.end(), (size_t)g.x * g.y * g.z, i);
    }
    if (tmax == 0 || owner.empty()) return cudaSuccess;
    char *base = (char *)scratch;
    unsigned *bar = (unsigned *)base;
    BatchItem<T, S> *d_items = (BatchItem<T, S> *)(base + 256);
    int *d_owner = (int *)(base + 256 + round_up((long long)n * sizeof(BatchItem<T, S>), 256));
    cudaError_t e = cudaMemsetAsync(bar, 0, 256, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_items, hi.data(), n * sizeof(BatchItem<T, S>), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_owner, owner.data(), owner.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    // the copies above read pageable host memory: finish them before the
    // host vectors go out of scope
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    const void *fn = rc ? (eq ? (const void *)batch_kernel<K, T, S, true, true>
                              : (const void *)batch_kernel<K, T, S, true, false>)
                        : (eq ? (const void *)batch_kernel<K, T, S, false, true>
                              : (const void *)batch_kernel<K, T, S, false, false>);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const dim3 blk = lb_block_batch(K);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, blk.x * blk.y * blk.z, 0)) !=
        cudaSuccess)
      return e;
    long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (grid > (long long)owner.size()) grid = (long long)owner.size();
    int nb = (int)owner.size();
    const BatchItem<T, S> *pi = d_items;
    const int *po = d_owner;
    unsigned long long lim = spins ? spins : kBarrierSpins;
    void *args[] = {(void *)&pi,   (void *)&n,   (void *)&po, (void *)&nb,
                    (void *)&tmax, (void *)&bar, (void *)&lim};
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), blk, args, 0, st);
  }
  // ---- single-pass step (D3Q19 only) ----
  static bool zprepare() {  // opt in to its dynamic shared memory, once
    if constexpr (K != 1) {
      return false;
    } else {
      static const bool ok =
          cudaFuncSetAttribute(zstep_kernel<T, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ZSmem<T>::total) == cudaSuccess &&
          cudaFuncSetAttribute(zstep_kernel<T, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ZSmem<T>::total) == cudaSuccess;
      return ok;
    }
  }
  static int zresident() {
    if constexpr (K != 1) {
      return 0;
    } else {
      int per_sm = 0;
      if (!zprepare() || cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &per_sm, zstep_kernel<T, S, false>, ZT_X * ZT_Y, ZSmem<T>::total) !=
                             cudaSuccess)
        return 0;
      return per_sm;
    }
  }
  static cudaError_t zstep(const LBRaw &r, const ZMaps &m, int zrun, cudaStream_t st) {
    if constexpr (K != 1) {
      return cudaErrorNotSupported;
    } else {
      if (!zprepare()) return cudaErrorInvalidValue;
      if (zrun < 1 || !z_tiles(r.nx, r.ny)) return cudaErrorInvalidValue;
      const dim3 grid(z_tiles_x(r.nx), z_tiles_y(r.ny), (r.nz + zrun - 1) / zrun),
          blk(ZT_X, ZT_Y, 1);
      if (r.p.rho_contrast)
        zstep_kernel<T, S, true><<<grid, blk, ZSmem<T>::total, st>>>(typed<T, S>(r), zrun, m.Q, m.U, m.C1);
      else
        zstep_kernel<T, S, false><<<grid, blk, ZSmem<T>::total, st>>>(typed<T, S>(r), zrun, m.Q, m.U, m.C1);
      return cudaGetLastError();
    }
  }
  static cudaError_t zpack(const LBRaw &r, void *Qz0, void *Qz1, void *Uz0, void *Uz1, void *C1z,
                           cudaStream_t st) {
    if constexpr (K != 1) {
      return cudaErrorNotSupported;
    } else {
      zpack_kernel<T, S><<<152 * 8, 256, 0, st>>>(typed<T, S>(r), (T *)Qz0, (T *)Qz1, (T *)Uz0,
                                                  (T *)Uz1, (T *)C1z, r.nxp, r.nyp);
      return cudaGetLastError();
    }
  }
  static cudaError_t zunpack(const LBRaw &r, const void *Qz, const void *Uz, void *Cout,
                             cudaStream_t st) {
    if constexpr (K != 1) {
      return cudaErrorNotSupported;
    } else {
      zunpack_kernel<T, S><<<152 * 8, 256, 0, st>>>(typed<T, S>(r), (const T *)Qz, (const T *)Uz,
                                                    (T *)Cout, r.nxp, r.nyp);
      return cudaGetLastError();
    }
  }
  static LBTable table() {
    LBTable t;
    t.zstep = &zstep;
    t.zresident = &zresident;
    t.zpack = &zpack;
    t.zunpack = &zunpack;
    t.batch = &batch;
    t.batch_bytes = &batch_bytes;
    t.moments = &moments;
    t.node = &node;
    t.init = &init;
    t.solid = &solid;
    t.get_pops = &get_pops;
    t.set_pops = &set_pops;
    t.materialize = &materialize;
    t.q = Lat<K>::Q;
    t.real_bytes = sizeof(T);
    t.store_bytes = sizeof(S);
    t.k16 = Store<S>::k16;
    return t;
  }
};

}  // namespace dsm
