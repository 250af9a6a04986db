// dsm_zstep.cuh -- the whole stage-2 lattice Boltzmann step (Sec. II.B) in one
// pass, for D3Q19 lattices that hold g as g_eq (tau_g = 1) with periodic faces.
// Included by dsm_lb_impl.cuh after the fused pass (node_body), whose per-node
// arithmetic it shares.
//
// The two-pass step reads the state twice: the moments pass rebuilds
// C(x) = sum_i g_eq_i(x - c_i) from the neighbours' (A, C, u), writes C, and the
// fused pass reads C back on the node's 1-neighbourhood for mu, G[C] and L[C].
// Here one block marches a 32 x 8 tile up a run of z planes and keeps this
// step's C on chip:
//   * the state's (A, u) and C of the last collision, and the solid C1, are
//     staged plane by plane into a shared ring by the tensor memory accelerator
//     (cp.async.bulk.tensor, one 3-D box per array and plane, completion on an
//     mbarrier per ring slot), two planes ahead of use;
//   * for plane z + 1 the block rebuilds this step's C on the tile and a one-node
//     halo (34 x 10 nodes) from the staged planes z .. z + 2 (the same per-node
//     sum as the moments pass, moments_eq_node) into a ring of four C planes;
//   * each thread then runs the fused pass (node_body) for its node of plane z
//     with C and C1 read from shared memory (ZIO below) and the populations f
//     pulled from global memory as in the two-pass step, and stores f, (A, u)
//     and its C.
// Per lattice update the step moves f in and out, (A, u, C) in and out and C1
// in: 196 B in FP32 instead of 172 + 24 B in two passes, and one launch.
//
// Layout.  (A, C, u_x, u_y) are interleaved per node as one 16-byte quad (one
// shared load serves every in-plane link of the sum), u_z has a plane of its
// own, and both, like C1, live in padded planes: 4 ghost columns on each x
// side (so that every box starts on a 16-byte boundary) and 2 ghost rows on
// each y side, which hold the periodic images of the edge nodes.  A box
// therefore never wraps; in z the ring simply loads plane z mod nz.  The
// collision writes each edge node's ghost copies as well.  Two such buffers
// (read, write) alternate from step to step.
#pragma once

#include <cuda.h>

namespace dsm {

constexpr int ZT_X = 32, ZT_Y = 8;                  // output tile (one node per thread)
constexpr int ZPAD_X = 4, ZPAD_Y = 2;               // ghost columns / rows per side
constexpr int ZB_X = ZT_X + 2 * ZPAD_X;             // staged box width (halo 2, x from -4)
constexpr int ZB_Y = ZT_Y + 2 * ZPAD_Y;             // staged quad / u_z box height (halo 2)
constexpr int ZB1_Y = ZT_Y + 2;                     // staged C1 box height (halo 1)
constexpr int ZC_X = ZT_X + 2, ZC_Y = ZT_Y + 2;     // this step's C: tile + halo 1
constexpr int Z_RING = 5;                           // staged planes (two ahead of use)
constexpr int Z_CRING = 4;                          // planes of this step's C kept (a power of 2)
constexpr long long kZWaitCycles = 4000000000ll;    // bounded mbarrier wait (~2 s)

template <class T>
struct alignas(4 * sizeof(T)) Quad {
  T v[4];
};

// Byte offsets of the shared-memory regions (each 128-byte aligned).
template <class T>
struct ZSmem {
  static constexpr size_t al(size_t b) { return (b + 127) / 128 * 128; }
  static constexpr size_t qbox = al(sizeof(T) * 4 * ZB_X * ZB_Y);  // (A, C, u_x, u_y)
  static constexpr size_t wbox = al(sizeof(T) * ZB_X * ZB_Y);      // u_z
  static constexpr size_t c1box = al(sizeof(T) * ZB_X * ZB1_Y);
  static constexpr size_t slot = qbox + wbox + c1box;
  static constexpr size_t cplane = al(sizeof(T) * ZC_X * ZC_Y);
  static constexpr size_t cring = Z_RING * slot;           // offset of the C ring
  static constexpr size_t bars = cring + Z_CRING * cplane;  // offset of the mbarriers
  static constexpr size_t total = bars + 8 * Z_RING;
  // bytes one ring slot receives from its three boxes
  static constexpr unsigned tx_bytes = sizeof(T) * (4 * ZB_X * ZB_Y + ZB_X * ZB_Y + ZB_X * ZB1_Y);
};

// Width and height of a padded plane: 4 ghost columns and 2 ghost rows on each
// side, the width rounded up to a multiple of 4 reals so that every row starts
// on a 16-byte boundary (the tensor maps' strides).  A lattice of any nx >= 32,
// ny >= 8 tiles into 32 x 8 blocks, the last ones ragged: their threads beyond
// the lattice take part in the rebuild and the barriers but run no pass, and
// boxes reaching past the padded planes read zeros (never used).
__host__ __device__ __forceinline__ int z_padded_x(int nx) { return (nx + 2 * ZPAD_X + 3) / 4 * 4; }
__host__ __device__ __forceinline__ int z_padded_y(int ny) { return ny + 2 * ZPAD_Y; }
__host__ __device__ __forceinline__ bool z_tiles(int nx, int ny) { return nx >= ZT_X && ny >= ZT_Y; }
__host__ __device__ __forceinline__ int z_tiles_x(int nx) { return (nx + ZT_X - 1) / ZT_X; }
__host__ __device__ __forceinline__ int z_tiles_y(int ny) { return (ny + ZT_Y - 1) / ZT_Y; }

// Padded index of node (x, y, z), x in [-ZPAD_X, nx + ZPAD_X), y in [-ZPAD_Y, ny + ZPAD_Y).
__host__ __device__ __forceinline__ long long zpidx(int x, int y, int z, int nxp, int nyp) {
  return ((long long)z * nyp + (y + ZPAD_Y)) * nxp + (x + ZPAD_X);
}

// ---- tensor-memory-accelerator and mbarrier primitives (inline PTX) ----------
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity to complete, for at most kZWaitCycles
// SM cycles; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kZWaitCycles) return false;
  return true;
}
// One 3-D box of a tensor map into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2),
      "r"(smem_addr(bar))
      : "memory");
}

// Dynamic shared memory of the single-pass step (the staged ring, the C ring
// and the mbarriers; layout in ZSmem).
extern __shared__ __align__(128) unsigned char zsm[];

// The fused pass's view of the neighbourhood in the single-pass step: this
// step's C from the C ring and C1 from the staged box, both in shared memory
// (byte offsets into zsm of the node's value in planes z - 1, z, z + 1); the
// quad (A, C, u_x, u_y) and u_z written to the padded output planes a.Qz,
// a.Uz, with the ghost copies of an edge node.  Wall links are fixed in an
// unrolled loop, and a solid node skips its f pulls (its C1 is at hand first).
template <class T>
struct ZIO {
  static constexpr bool kUnrollWall = true;
  static constexpr bool kSolidFirst = true;
  unsigned co[3], c1o[3];
  int x, y, z;
  template <class L, class T_, class S>
  __device__ __forceinline__ T C(const LBArgs<T_, S> &, const Hood &, int i) const {
    return *reinterpret_cast<const T *>(zsm + co[L::cz(i) + 1] +
                                        sizeof(T) * (L::cy(i) * ZC_X + L::cx(i)));
  }
  template <class L, class T_, class S>
  __device__ __forceinline__ T C1(const LBArgs<T_, S> &, const Hood &, int i) const {
    return *reinterpret_cast<const T *>(zsm + c1o[L::cz(i) + 1] +
                                        sizeof(T) * (L::cy(i) * ZB_X + L::cx(i)));
  }
  template <class L, class S>
  __device__ __forceinline__ void put_eq(const LBArgs<T, S> &a, int, T c, T A, T ux, T uy,
                                         T uz) const {
    Quad<T> m;
    m.v[0] = A;
    m.v[1] = c;
    m.v[2] = ux;
    m.v[3] = uy;
    const long long q = zpidx(x, y, z, a.nxp, a.nyp);
    const long long gx = x < 2 ? a.nx : (x >= a.nx - 2 ? -a.nx : 0);
    const long long gy = (long long)(y < 2 ? a.ny : (y >= a.ny - 2 ? -a.ny : 0)) * a.nxp;
    const long long P = (long long)a.nxp * a.nyp * a.nz;  // padded nodes (checked build)
    auto put1 = [&](long long p) {
      p = chk(a.err, p, P);
      *reinterpret_cast<Quad<T> *>(a.Qz + 4 * p) = m;
      a.Uz[p] = uz;
    };
    put1(q);
    if (gx) put1(q + gx);
    if (gy) put1(q + gy);
    if (gx && gy) put1(q + gx + gy);
  }
};

// K2z: one step.  Grid (ceil(nx / 32), ceil(ny / 8), ceil(nz / zrun)); block 32 x 8;
// a.Qz / a.Uz receive this step's quads (A, C, u_x, u_y) and u_z.  tmQ: the
// padded quads of the state, as a 3-D tensor (4 nxp, nyp, nz); tmU: its u_z
// (nxp, nyp, nz); tmC1: padded C1 (nxp, nyp, nz).
template <class T, class S, bool RC>
__global__ void __launch_bounds__(ZT_X *ZT_Y, sizeof(T) == 8 ? 1 : 3)
    zstep_kernel(LBArgs<T, S> a, int zrun, const __grid_constant__ CUtensorMap tmQ,
                 const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmC1) {
  using L = Lat<1>;
  using SM = ZSmem<T>;
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(zsm + SM::bars);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ZT_X * ty;
  const int nz = a.nz;
  const int x0 = blockIdx.x * ZT_X, y0 = blockIdx.y * ZT_Y;
  const int z0 = blockIdx.z * zrun, z1 = min(z0 + zrun, nz);
  // staged plane p has ring index k = p - (z0 - 2); the run stages z0 - 2 .. z1 + 1
  const int nk = z1 - z0 + 4;
  auto slot_of = [&](int k) { return (unsigned)((k % Z_RING) * SM::slot); };
  auto issue = [&](int k) {  // one thread: stage plane z0 - 2 + k into its ring slot
    if (k >= nk) return;
    int pz = (z0 - 2 + k) % nz;
    if (pz < 0) pz += nz;
    unsigned char *s = zsm + slot_of(k);
    unsigned long long *b = bar + k % Z_RING;
    mbar_expect_tx(b, SM::tx_bytes);
    tma_load_3d(s, &tmQ, 4 * x0, y0, pz, b);
    tma_load_3d(s + SM::qbox, &tmU, x0, y0, pz, b);
    tma_load_3d(s + SM::qbox + SM::wbox, &tmC1, x0, y0 + 1, pz, b);
  };
  if (tid == 0) {
    for (int s = 0; s < Z_RING; s++) mbar_init(bar + s, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0)
    for (int k = 0; k < Z_RING; k++) issue(k);
  // every thread waits on every staged plane, in order; kw: the first plane
  // this thread has not seen arrive; late: a plane did not arrive in time
  int kw = 0;
  bool late = false;
  auto wait_to = [&](int k) {  // staged planes up to k have arrived
    for (; !late && kw <= k; kw++)
      if (!mbar_wait_bounded(bar + kw % Z_RING, (unsigned)(kw / Z_RING) & 1u)) late = true;
  };
  // this step's C on the tile and its halo for plane q, from staged planes
  // q - 1, q, q + 1 (ring indices q - z0 + 1 .. q - z0 + 3)
  // the C nodes this thread rebuilds: c = tid and, for the first 84 threads,
  // c = tid + 256; node (cx - 1, cy - 1) of the tile sits at (cx + 3, cy + 1)
  // in the boxes (byte offsets of its quad and of its u_z)
  const int nc = tid + ZT_X * ZT_Y < ZC_X * ZC_Y ? 2 : 1;
  unsigned bq[2], bw[2];
#pragma unroll
  for (int r = 0; r < 2; r++) {
    const int c = tid + r * ZT_X * ZT_Y;
    const int bo = (c / ZC_X + 1) * ZB_X + (c % ZC_X + 3);
    bq[r] = (unsigned)(sizeof(Quad<T>) * bo);
    bw[r] = (unsigned)(SM::qbox + sizeof(T) * bo);
  }
  // (m0, m1, m2: byte offsets of the ring slots of staged planes q - 1, q,
  // q + 1; cdst: that of this step's C of plane q)
  auto rebuild_c = [&](unsigned m0, unsigned m1, unsigned m2, unsigned cdst) {
    T *dst = reinterpret_cast<T *>(zsm + cdst);
    for (int r = 0; r < nc; r++) {
      T Ay[L::Q], Cy[L::Q], uy[L::Q][3];
#pragma unroll
      for (int i = 0; i < L::Q; i++) {
        // x - c_i in plane q - c_z: a constant step from the C node's offsets
        const unsigned sl = L::cz(i) > 0 ? m0 : (L::cz(i) < 0 ? m2 : m1);
        const int step = -(L::cy(i) * ZB_X + L::cx(i));
        const Quad<T> m = *reinterpret_cast<const Quad<T> *>(zsm + sl + bq[r] +
                                                             (int)sizeof(Quad<T>) * step);
        Ay[i] = m.v[0];
        Cy[i] = m.v[1];
        uy[i][0] = (i == 0 || L::cx(i)) ? m.v[2] : T(0);
        uy[i][1] = (i == 0 || L::cy(i)) ? m.v[3] : T(0);
        uy[i][2] = (i == 0 || L::cz(i))
                       ? *reinterpret_cast<const T *>(zsm + sl + bw[r] + (int)sizeof(T) * step)
                       : T(0);
      }
      dst[tid + r * ZT_X * ZT_Y] = moments_eq_node<L, T>(Ay, Cy, uy);
    }
  };
  // prologue: this step's C of planes z0 - 1 and z0 (staged planes z0 - 2 ..
  // z0 + 1 in slots 0 .. 3; C ring slots 0, 1)
  wait_to(3);
  if (!late) {
    rebuild_c(0 * SM::slot, 1 * SM::slot, 2 * SM::slot, SM::cring);
    rebuild_c(1 * SM::slot, 2 * SM::slot, 3 * SM::slot, SM::cring + SM::cplane);
  }
  ZIO<T> io;
  io.x = x0 + tx;
  io.y = y0 + ty;
  const bool inside = io.x < a.nx && io.y < a.ny;  // ragged last tiles
  // ring positions at plane z, advanced by one each plane: sk, the slot of
  // staged plane z - 1; cq, the C ring slot of plane z - 1
  auto next5 = [](int v) { return v + 1 == Z_RING ? 0 : v + 1; };
  int sk = 1, cq = 0;
  const unsigned node_c = sizeof(T) * ((ty + 1) * ZC_X + (tx + 1));
  const unsigned node_c1 = (unsigned)(SM::qbox + SM::wbox) + sizeof(T) * ((ty + 1) * ZB_X + (tx + ZPAD_X));
  for (int z = z0; z < z1; z++) {
    const int s0 = sk, s1 = next5(s0), s2 = next5(s1), s3 = next5(s2);
    wait_to(z - z0 + 4);  // staged plane z + 2
    if (!late)
      rebuild_c(s1 * SM::slot, s2 * SM::slot, s3 * SM::slot,
                SM::cring + ((cq + 2) & (Z_CRING - 1)) * SM::cplane);
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
    for (int d = 0; d < 3; d++)
      io.co[d] = (unsigned)(SM::cring + ((cq + d) & (Z_CRING - 1)) * SM::cplane) + node_c;
    io.c1o[0] = s0 * SM::slot + node_c1;
    io.c1o[1] = s1 * SM::slot + node_c1;
    io.c1o[2] = s2 * SM::slot + node_c1;
    io.z = z;
    node_body<1, T, S, 2, MODE_STEP, RC, true, false, ZIO<T>>(a, io.x, io.y, z, inside, 0, io);
    sk = s1;
    cq = (cq + 1) & (Z_CRING - 1);
  }
}

// Canonical g_eq state (A, u planes, C of the last collision) and C1 -> the
// padded buffers of the single-pass step (both buffers, so that every ghost
// position holds a finite value), over every padded position.
template <class T, class S>
__global__ void __launch_bounds__(256) zpack_kernel(LBArgs<T, S> a, T *Qz0, T *Qz1, T *Uz0, T *Uz1,
                                                    T *C1z, int nxp, int nyp) {
  const long long P = (long long)nxp * nyp * a.nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < P;
       q += (long long)gridDim.x * blockDim.x) {
    const int px = (int)(q % nxp), py = (int)((q / nxp) % nyp), z = (int)(q / ((long long)nxp * nyp));
    int x = (px - ZPAD_X) % a.nx, y = (py - ZPAD_Y) % a.ny;
    if (x < 0) x += a.nx;
    if (y < 0) y += a.ny;
    const long long n = x + (long long)a.nx * (y + (long long)a.ny * z);
    Quad<T> m;
    m.v[0] = a.Mp[0][n];
    m.v[1] = a.Cprev[n];
    m.v[2] = a.Mp[1][n];
    m.v[3] = a.Mp[2][n];
    reinterpret_cast<Quad<T> *>(Qz0)[q] = m;
    reinterpret_cast<Quad<T> *>(Qz1)[q] = m;
    Uz0[q] = a.Mp[3][n];
    Uz1[q] = a.Mp[3][n];
    C1z[q] = a.C1[n];
  }
}

// Padded buffers -> canonical g_eq state (A, u planes and C of the last collision).
template <class T, class S>
__global__ void __launch_bounds__(256) zunpack_kernel(LBArgs<T, S> a, const T *Qz, const T *Uz,
                                                      T *Cout, int nxp, int nyp) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % a.nx), y = (int)((n / a.nx) % a.ny), z = (int)(n / ((long long)a.nx * a.ny));
    const long long q = zpidx(x, y, z, nxp, nyp);
    const Quad<T> m = reinterpret_cast<const Quad<T> *>(Qz)[q];
    a.Mp[0][n] = m.v[0];
    Cout[n] = m.v[1];
    a.Mp[1][n] = m.v[2];
    a.Mp[2][n] = m.v[3];
    a.Mp[3][n] = Uz[q];
  }
}

}  // namespace dsm
