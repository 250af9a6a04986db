// dsm_mlz.cuh -- the N-fluid lattice Boltzmann step (Sec. II.B for N + 1
// components) in one pass, for D3Q19 lattices that hold every g_f as g_eq
// (tau_g = 1) with periodic faces.  Included by dsm_multi.cu after the N-fluid
// fused pass (ml_node_body), whose per-node arithmetic it shares; the ring,
// the tensor-memory-accelerator loads and the bounded waits are those of the
// two-fluid single-pass step (dsm_zstep.cuh).
//
// The two-pass N-fluid step reads the state twice: a moments pass per free
// fluid rebuilds C_f(x) = sum_i g_eq_i(x - c_i) from the neighbours'
// (A_f, C_f, u), and the fused pass reads C1 and every C_f back on the node's
// 1-neighbourhood (57 scattered loads per node for three fluids).  Here one
// block marches a 32 x 8 tile up a run of z planes:
//   * per plane, the state's quad (A_1, C_1, u_x, u_y), u_z, one pair
//     (A_f, C_f) per further free fluid and the solid C1 are staged into a
//     five-slot shared ring by cp.async.bulk.tensor, two planes ahead of use;
//   * for plane z + 1 the block rebuilds this step's C_f of every free fluid
//     on the tile and a one-node halo (34 x 10 nodes; u read once for all
//     fluids) into a ring of four C planes per fluid;
//   * each thread runs the N-fluid fused pass for its node of plane z with C1
//     and every C_f from shared memory, pulls f from global memory, and stores
//     f, the quad, u_z and the pairs (with the ghost copies of an edge node).
// Per lattice update the step moves f in and out (152 B in FP32), the state
// (A_f, C_f per free fluid and u) in and out, and C1 in: 212 B for three
// fluids, 228 B for four, in one launch.
//
// Layout: as in the two-fluid step, padded planes (4 ghost columns on each x
// side, 2 ghost rows on each y side) holding the periodic images of the edge
// nodes; the pairs of the free fluids 2 .. NF are stacked along z in one
// buffer (fluid e at planes (e - 1) nz .. e nz - 1), so that one tensor map
// serves all of them.  Two such buffers (read, write) alternate.
#pragma once

namespace dsm {

template <class T>
struct alignas(2 * sizeof(T)) Pair {
  T v[2];
};

// Byte offsets of the shared-memory regions of the N-fluid single-pass step
// (each 128-byte aligned): per ring slot the quad box, the u_z box, NF - 1
// pair boxes and the C1 box; the C ring (Z_CRING slots of NF planes); the
// mbarriers.
template <class T, int NF>
struct MLZSmem {
  static constexpr size_t al(size_t b) { return (b + 127) / 128 * 128; }
  static constexpr size_t qbox = al(sizeof(T) * 4 * ZB_X * ZB_Y);
  static constexpr size_t wbox = al(sizeof(T) * ZB_X * ZB_Y);
  static constexpr size_t pbox = al(sizeof(T) * 2 * ZB_X * ZB_Y);
  static constexpr size_t c1box = al(sizeof(T) * ZB_X * ZB1_Y);
  static constexpr size_t woff = qbox;
  static constexpr size_t poff = woff + wbox;
  static constexpr size_t c1off = poff + (NF - 1) * pbox;
  static constexpr size_t slot = c1off + c1box;
  static constexpr size_t cplane = al(sizeof(T) * ZC_X * ZC_Y);
  static constexpr size_t cring = Z_RING * slot;
  static constexpr size_t bars = cring + Z_CRING * NF * cplane;
  static constexpr size_t total = bars + 8 * Z_RING;
  static constexpr unsigned tx_bytes =
      sizeof(T) * (4 * ZB_X * ZB_Y + ZB_X * ZB_Y + (NF - 1) * 2 * ZB_X * ZB_Y + ZB_X * ZB1_Y);
};

// The N-fluid fused pass's view in the single-pass step: this step's C_f from
// the C ring and C1 from the staged box, both in shared memory (co, c1o: byte
// offsets into zsm of the node's value in planes z - 1, z, z + 1; fluid f's
// C plane follows fluid 0's at f * cplane); the state to the padded output
// buffers a.Qz, a.Uz, a.Pz with the ghost copies of an edge node.
template <class T, int NF>
struct MLZIO {
  static constexpr bool kSolidFirst = true;
  static constexpr bool kZ = true;
  static constexpr bool kUnrollWall = true;
  unsigned co[3], c1o[3];
  int x, y, z;
  template <class L>
  __device__ __forceinline__ T C1(const MLArgs<T> &, const Hood &, int, int i) const {
    return *reinterpret_cast<const T *>(zsm + c1o[L::cz(i) + 1] +
                                        sizeof(T) * (L::cy(i) * ZB_X + L::cx(i)));
  }
  template <class L>
  __device__ __forceinline__ T C(const MLArgs<T> &, const Hood &, int, int f, int i) const {
    return *reinterpret_cast<const T *>(zsm + co[L::cz(i) + 1] + f * MLZSmem<T, NF>::cplane +
                                        sizeof(T) * (L::cy(i) * ZC_X + L::cx(i)));
  }
  template <class L, int NF_>
  __device__ __forceinline__ void put_eq(const MLArgs<T> &a, long long, const T (&A)[NF_],
                                         const T (&C)[NF_], const T (&u)[3]) const {
    static_assert(NF_ == NF, "one pair per further free fluid");
    Quad<T> m;
    m.v[0] = A[0];
    m.v[1] = C[0];
    m.v[2] = u[0];
    m.v[3] = u[1];
    Pair<T> pr[NF > 1 ? NF - 1 : 1];
#pragma unroll
    for (int e = 1; e < NF; e++) {
      pr[e - 1].v[0] = A[e];
      pr[e - 1].v[1] = C[e];
    }
    const long long P = (long long)a.nxp * a.nyp * a.nz;  // one padded buffer plane set
    const long long q = zpidx(x, y, z, a.nxp, a.nyp);
    const long long gx = x < 2 ? a.nx : (x >= a.nx - 2 ? -a.nx : 0);
    const long long gy = (long long)(y < 2 ? a.ny : (y >= a.ny - 2 ? -a.ny : 0)) * a.nxp;
    auto put1 = [&](long long p) {
      p = chk(a.err, p, P);  // (checked build)
      *reinterpret_cast<Quad<T> *>(a.Qz + 4 * p) = m;
      a.Uz[p] = u[2];
#pragma unroll
      for (int e = 1; e < NF; e++)
        *reinterpret_cast<Pair<T> *>(a.Pz + 2 * ((e - 1) * P + p)) = pr[e - 1];
    };
    put1(q);
    if (gx) put1(q + gx);
    if (gy) put1(q + gy);
    if (gx && gy) put1(q + gx + gy);
  }
};

// One N-fluid step.  Grid (ceil(nx / 32), ceil(ny / 8), ceil(nz / zrun)); block
// 32 x 8 (threads of a ragged last tile beyond the lattice run no pass);
// a.Qz / a.Uz / a.Pz receive this step's state.  tmQ: the padded quads of
// the state (4 nxp, nyp, nz); tmU: its u_z (nxp, nyp, nz); tmP: its pairs
// (2 nxp, nyp, (NF - 1) nz; any valid map when NF = 1); tmC1: padded C1.
// RCV: the fluids' densities may differ (else the density map is compiled out).
template <class T, int NF, bool RCV>
__global__ void __launch_bounds__(ZT_X *ZT_Y, sizeof(T) == 8 ? 1 : 2)
    mlz_kernel(MLArgs<T> a, int zrun, const __grid_constant__ CUtensorMap tmQ,
               const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmP,
               const __grid_constant__ CUtensorMap tmC1) {
  using L = Lat<1>;
  using SM = MLZSmem<T, NF>;
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(zsm + SM::bars);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ZT_X * ty;
  const int nz = a.nz;
  const int x0 = blockIdx.x * ZT_X, y0 = blockIdx.y * ZT_Y;
  const int z0 = blockIdx.z * zrun, z1 = min(z0 + zrun, nz);
  // staged plane p has ring index k = p - (z0 - 2); the run stages z0 - 2 .. z1 + 1
  const int nk = z1 - z0 + 4;
  auto issue = [&](int k) {  // one thread: stage plane z0 - 2 + k into its ring slot
    if (k >= nk) return;
    int pz = (z0 - 2 + k) % nz;
    if (pz < 0) pz += nz;
    unsigned char *s = zsm + (k % Z_RING) * SM::slot;
    unsigned long long *b = bar + k % Z_RING;
    mbar_expect_tx(b, SM::tx_bytes);
    tma_load_3d(s, &tmQ, 4 * x0, y0, pz, b);
    tma_load_3d(s + SM::woff, &tmU, x0, y0, pz, b);
#pragma unroll
    for (int e = 1; e < NF; e++)
      tma_load_3d(s + SM::poff + (e - 1) * SM::pbox, &tmP, 2 * x0, y0, (e - 1) * nz + pz, b);
    tma_load_3d(s + SM::c1off, &tmC1, x0, y0 + 1, pz, b);
  };
  if (tid == 0) {
    for (int s = 0; s < Z_RING; s++) mbar_init(bar + s, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0)
    for (int k = 0; k < Z_RING; k++) issue(k);
  int kw = 0;
  bool late = false;
  auto wait_to = [&](int k) {  // staged planes up to k have arrived
    for (; !late && kw <= k; kw++)
      if (!mbar_wait_bounded(bar + kw % Z_RING, (unsigned)(kw / Z_RING) & 1u)) late = true;
  };
  // the C nodes this thread rebuilds: c = tid and, for the first 84 threads,
  // c = tid + 256; node (cx - 1, cy - 1) of the tile sits at box index
  // bo = (cy + 1) ZB_X + cx + 3
  const int nc = tid + ZT_X * ZT_Y < ZC_X * ZC_Y ? 2 : 1;
  int bo[2];
#pragma unroll
  for (int r = 0; r < 2; r++) {
    const int c = tid + r * ZT_X * ZT_Y;
    bo[r] = (c / ZC_X + 1) * ZB_X + (c % ZC_X + 3);
  }
  // this step's C_f of every free fluid on the tile and its halo for plane q,
  // from staged planes q - 1, q, q + 1 (ring byte offsets m0, m1, m2) into the
  // C ring slot at byte offset cdst: per node the two-fluid moments sum
  // (moments_eq_node), with u read once for all fluids
  auto rebuild_c = [&](unsigned m0, unsigned m1, unsigned m2, unsigned cdst) {
    for (int r = 0; r < nc; r++) {
      // the staged values of link i at x - c_i: A_f, C_f, u (u_z only where
      // c_i has a z component, or at the node itself)
      auto link = [&](int i, T (&Af)[NF], T (&Cf)[NF], T (&ul)[3]) {
        const unsigned sl = L::cz(i) > 0 ? m0 : (L::cz(i) < 0 ? m2 : m1);
        const int p = bo[r] - (L::cy(i) * ZB_X + L::cx(i));  // box index of x - c_i
        const Quad<T> m = *reinterpret_cast<const Quad<T> *>(zsm + sl + sizeof(Quad<T>) * p);
        ul[0] = m.v[2];
        ul[1] = m.v[3];
        ul[2] = (i == 0 || L::cz(i))
                    ? *reinterpret_cast<const T *>(zsm + sl + SM::woff + sizeof(T) * p)
                    : T(0);
        Af[0] = m.v[0];
        Cf[0] = m.v[1];
#pragma unroll
        for (int e = 1; e < NF; e++) {
          const Pair<T> q = *reinterpret_cast<const Pair<T> *>(
              zsm + sl + SM::poff + (e - 1) * SM::pbox + sizeof(Pair<T>) * p);
          Af[e] = q.v[0];
          Cf[e] = q.v[1];
        }
      };
      T A0[NF], C0[NF], u0[3];
      link(0, A0, C0, u0);
      // opposite links (i, i + 1) of one weight as one pair: c.u and
      // cu (3 + 9/2 cu) once for every fluid, then A + C t per fluid
      // (moments_eq_node's arithmetic, paired; dsm_pair.cuh)
      Pr<T> sa[NF], sd[NF];
#pragma unroll
      for (int f = 0; f < NF; f++) sa[f] = sd[f] = pr(T(0), T(0));
#pragma unroll
      for (int i = 1; i < L::Q; i += 2) {
        T Ai[NF], Ci[NF], ui[3], Ab[NF], Cb[NF], ub[3];
        link(i, Ai, Ci, ui);
        link(i + 1, Ab, Cb, ub);
        const Pr<T> cu = pr(cdot<L>(i, ui[0], ui[1], ui[2]), cdot<L>(i + 1, ub[0], ub[1], ub[2]));
        const Pr<T> t = pr_mul(cu, pr_fma(pr(T(4.5), T(4.5)), cu, pr(T(3), T(3))));
#pragma unroll
        for (int f = 0; f < NF; f++) {
          const Pr<T> v = pr_fma(pr(Ci[f], Cb[f]), t, pr(Ai[f], Ab[f]));
          if (L::w(i) == L::w(1)) sa[f] = pr_add(sa[f], v);
          else sd[f] = pr_add(sd[f], v);
        }
      }
      const T uu0 = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2];
#pragma unroll
      for (int f = 0; f < NF; f++) {
        const T out = T(1.0 - L::w(0)) * A0[f] + T(1.5) * C0[f] * uu0;
        const T saf = sa[f].a + sa[f].b, sdf = sd[f].a + sd[f].b;
        reinterpret_cast<T *>(zsm + cdst + f * SM::cplane)[tid + r * ZT_X * ZT_Y] =
            C0[f] + ((T(L::w(1)) * saf + T(L::w(L::Q - 1)) * sdf) - out);
      }
    }
  };
  auto cslot = [&](int c) { return (unsigned)(SM::cring + c * NF * SM::cplane); };
  // prologue: this step's C of planes z0 - 1 and z0 (staged planes z0 - 2 ..
  // z0 + 1 in slots 0 .. 3; C ring slots 0, 1)
  wait_to(3);
  if (!late) {
    rebuild_c(0 * SM::slot, 1 * SM::slot, 2 * SM::slot, cslot(0));
    rebuild_c(1 * SM::slot, 2 * SM::slot, 3 * SM::slot, cslot(1));
  }
  MLZIO<T, NF> io;
  io.x = x0 + tx;
  io.y = y0 + ty;
  auto next5 = [](int v) { return v + 1 == Z_RING ? 0 : v + 1; };
  int sk = 1, cq = 0;  // ring slots of staged plane z - 1 and of C plane z - 1
  const unsigned node_c = sizeof(T) * ((ty + 1) * ZC_X + (tx + 1));
  const unsigned node_c1 = (unsigned)SM::c1off + sizeof(T) * ((ty + 1) * ZB_X + (tx + ZPAD_X));
  for (int z = z0; z < z1; z++) {
    const int s0 = sk, s1 = next5(s0), s2 = next5(s1), s3 = next5(s2);
    wait_to(z - z0 + 4);  // staged plane z + 2
    if (!late)
      rebuild_c(s1 * SM::slot, s2 * SM::slot, s3 * SM::slot, cslot((cq + 2) & (Z_CRING - 1)));
    // this step's C of plane z + 1 is complete, and staged plane z - 2 is free
    if (__syncthreads_or(late)) {
      // a staged plane did not arrive: latch the error, wait (again bounded)
      // for the copies still in flight so that none outlives the block, return
      if (tid == 0) {
        atomicOr(a.err, ERR_TIMEOUT);
        const int issued = min(z - z0 + Z_RING, nk);
        for (int k = kw; k < issued; k++)
          mbar_wait_bounded(bar + k % Z_RING, (unsigned)(k / Z_RING) & 1u);
      }
      return;
    }
    if (tid == 0) issue(z - z0 + Z_RING);
#pragma unroll
    for (int d = 0; d < 3; d++) io.co[d] = cslot((cq + d) & (Z_CRING - 1)) + node_c;
    io.c1o[0] = s0 * SM::slot + node_c1;
    io.c1o[1] = s1 * SM::slot + node_c1;
    io.c1o[2] = s2 * SM::slot + node_c1;
    io.z = z;
    ml_node_body<1, T, NF, ML_STEP, true, false, MLZIO<T, NF>, RCV>(a, io.x, io.y, z, io);
    sk = s1;
    cq = (cq + 1) & (Z_CRING - 1);
  }
}

// Canonical g_eq state (A_f, u planes, C_f of the last collision) and C1 ->
// both padded buffers (so that every ghost position holds a finite value).
template <class T, int NF>
__global__ void __launch_bounds__(256) mlz_pack_kernel(MLArgs<T> a, T *Qz0, T *Qz1, T *Uz0,
                                                       T *Uz1, T *Pz0, T *Pz1, T *C1z) {
  const int nxp = a.nxp, nyp = a.nyp;
  const long long P = (long long)nxp * nyp * a.nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < P;
       q += (long long)gridDim.x * blockDim.x) {
    const int px = (int)(q % nxp), py = (int)((q / nxp) % nyp), z = (int)(q / ((long long)nxp * nyp));
    int x = (px - ZPAD_X) % a.nx, y = (py - ZPAD_Y) % a.ny;
    if (x < 0) x += a.nx;
    if (y < 0) y += a.ny;
    const long long n = x + (long long)a.nx * (y + (long long)a.ny * z);
    Quad<T> m;
    m.v[0] = a.A[n];
    m.v[1] = a.Cprev[n];
    m.v[2] = a.U[n];
    m.v[3] = a.U[a.pitch + n];
    reinterpret_cast<Quad<T> *>(Qz0)[q] = m;
    reinterpret_cast<Quad<T> *>(Qz1)[q] = m;
    Uz0[q] = a.U[2 * a.pitch + n];
    Uz1[q] = a.U[2 * a.pitch + n];
    for (int e = 1; e < NF; e++) {
      Pair<T> pr;
      pr.v[0] = a.A[e * a.pitch + n];
      pr.v[1] = a.Cprev[e * a.pitch + n];
      reinterpret_cast<Pair<T> *>(Pz0)[(e - 1) * P + q] = pr;
      reinterpret_cast<Pair<T> *>(Pz1)[(e - 1) * P + q] = pr;
    }
    C1z[q] = a.C1[n];
  }
}

// Padded buffers -> canonical g_eq state (A_f, u planes and, into Cout, C_f of
// the last collision).
template <class T, int NF>
__global__ void __launch_bounds__(256) mlz_unpack_kernel(MLArgs<T> a, const T *Qz, const T *Uz,
                                                         const T *Pz, T *Cout) {
  const long long P = (long long)a.nxp * a.nyp * a.nz;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % a.nx), y = (int)((n / a.nx) % a.ny), z = (int)(n / ((long long)a.nx * a.ny));
    const long long q = zpidx(x, y, z, a.nxp, a.nyp);
    const Quad<T> m = reinterpret_cast<const Quad<T> *>(Qz)[q];
    a.A[n] = m.v[0];
    Cout[n] = m.v[1];
    a.U[n] = m.v[2];
    a.U[a.pitch + n] = m.v[3];
    a.U[2 * a.pitch + n] = Uz[q];
    for (int e = 1; e < NF; e++) {
      const Pair<T> pr = reinterpret_cast<const Pair<T> *>(Pz)[(e - 1) * P + q];
      a.A[e * a.pitch + n] = pr.v[0];
      Cout[e * a.pitch + n] = pr.v[1];
    }
  }
}

}  // namespace dsm
