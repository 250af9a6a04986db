// dsm_common.cuh -- lattice tables, storage codecs and kernel arguments shared
// by the CUDA kernels of libdsm (sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dsm.h"

namespace dsm {

constexpr int QMAX = 19;

// --------------------------------------------------------------------------
// Lattices.  D2Q9: the velocity/weight table printed in Sec. II.B of the
// paper.  D3Q19: textbook set (rest 1/3, six axis links 1/18, twelve face
// diagonals 1/36), opposite directions adjacent (1,2), (3,4), ...
// --------------------------------------------------------------------------
template <int K>
struct Lat;

template <>
struct Lat<0> {
  static constexpr int Q = 9;
  static constexpr int D = 2;
  __host__ __device__ static constexpr int cx(int i) {
    return i == 1 || i == 5 || i == 7 ? 1 : (i == 2 || i == 6 || i == 8 ? -1 : 0);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return i == 3 || i == 5 || i == 8 ? 1 : (i == 4 || i == 6 || i == 7 ? -1 : 0);
  }
  __host__ __device__ static constexpr int cz(int) { return 0; }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : (i == 1 ? 2 : i == 2 ? 1 : i == 3 ? 4 : i == 4 ? 3 : i == 5 ? 6
                                                    : i == 6 ? 5 : i == 7 ? 8 : 7);
  }
};

template <>
struct Lat<1> {
  static constexpr int Q = 19;
  static constexpr int D = 3;
  // 0 rest; 1..6 axis (+x,-x,+y,-y,+z,-z); 7..18 face diagonals in +- pairs
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
  }
};

// Index of the direction (cx, cy, cz) in lattice L (0 if absent).
template <class L>
__host__ __device__ constexpr int lat_index(int cx, int cy, int cz) {
  int k = 0;
  for (int i = 1; i < L::Q; i++)
    if (L::cx(i) == cx && L::cy(i) == cy && L::cz(i) == cz) k = i;
  return k;
}

// --------------------------------------------------------------------------
// Population storage.  For the 16-bit precisions the hydrodynamic population is
// stored as its offset from the rest weight, f_i - w_i, and the order-parameter
// populations g_i (i != 0) as they are; g_0 lives in a separate FP32 array so
// that the local mass can be kept exact (see the fused kernel).
// --------------------------------------------------------------------------
template <class S>
struct Store;

template <>
struct Store<double> {
  static constexpr bool k16 = false;
  __device__ static double dec(double v) { return v; }
  __device__ static double enc(double v) { return v; }
};
template <>
struct Store<float> {
  static constexpr bool k16 = false;
  __device__ static float dec(float v) { return v; }
  __device__ static float enc(float v) { return v; }
};
template <>
struct Store<__nv_bfloat16> {
  static constexpr bool k16 = true;
  __device__ static float dec(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __nv_bfloat16 enc(float v) { return __float2bfloat16_rn(v); }
};
// FP16 stores its values scaled by 2^10: population offsets f_i - w_i and
// small g_i (1e-6 .. 1e-4) would otherwise fall in FP16's subnormal range; the
// largest stored magnitudes (~0.06) stay far below its 65504 limit.  Scaling by
// a power of two adds no rounding.
template <>
struct Store<__half> {
  static constexpr bool k16 = true;
  __device__ static float dec(__half v) { return __half2float(v) * (1.0f / 1024.0f); }
  __device__ static __half enc(float v) { return __float2half_rn(v * 1024.0f); }
};

// Scalar parameters of the step, precomputed on the host.
struct StepParams {
  double kappa1, kappa2, kappa3;
  double a2;                // alpha^2
  double alpha_s;           // width of the solid tanh profile (Bouzidi distance)
  double rho2, rho3, tau2, tau3, tau_g;
  double body[3];
  double beta, omega;
  int rho_contrast;         // rho2 != rho3
  int face[6];              // x-, x+, y-, y+, z-, z+: 0 periodic, 1 mirror, 2 wall
  int walls;                // some face is not periodic
};

// The same constants in the arithmetic type T, with every product and
// reciprocal the kernels need formed once on the host: no double-precision
// conversion or division is left in the FP32 kernels.
template <class T>
struct ConstT {
  T k2, k3, a2k2, a2k3, k13, a2k13;  // kappa_2, kappa_3, a^2 kappa_n, kappa_1 + kappa_3
  T alpha_s;
  T rho2, rho3, drho, inv_rho3;      // densities, rho2 - rho3, 1/rho3
  T tau2, tau3, om2, om3, omg;       // relaxation times and 1/tau2, 1/tau3, 1/tau_g
  T body[3];
  T beta2, omega2;                   // 2 beta, 2 Omega
  static ConstT make(const StepParams &p) {
    ConstT c;
    c.k2 = T(p.kappa2); c.k3 = T(p.kappa3);
    c.a2k2 = T(p.a2 * p.kappa2); c.a2k3 = T(p.a2 * p.kappa3);
    c.k13 = T(p.kappa1 + p.kappa3); c.a2k13 = T(p.a2 * (p.kappa1 + p.kappa3));
    c.alpha_s = T(p.alpha_s);
    c.rho2 = T(p.rho2); c.rho3 = T(p.rho3); c.drho = T(p.rho2 - p.rho3); c.inv_rho3 = T(1.0 / p.rho3);
    c.tau2 = T(p.tau2); c.tau3 = T(p.tau3);
    c.om2 = T(1.0 / p.tau2); c.om3 = T(1.0 / p.tau3); c.omg = T(1.0 / p.tau_g);
    for (int a = 0; a < 3; a++) c.body[a] = T(p.body[a]);
    c.beta2 = T(2.0 * p.beta); c.omega2 = T(2.0 * p.omega);
    return c;
  }
};

// Pointers and sizes of one lattice for the LB kernels.
template <class T, class S>
struct LBArgs {
  int nx, ny, nz;
  long long N;       // nx*ny*nz
  long long pitch;   // population plane stride (elements), >= N, multiple of 64
  const S *f_in;
  const S *g_in;
  const float *g0_in;  // 16-bit precisions: FP32 g_0 (else unused)
  S *f_out;
  S *g_out;
  float *g0_out;
  T *C;                // concentration (moments pass output)
  const T *Cprev;      // concentration of the state's last collision (g held as g_eq)
  const T *C1;         // frozen solid (stage 2)
  const unsigned char *mask;  // solid region S (stage 1)
  T *fields;           // FIELDS mode output: 10 x N
  double *partials;    // OBS mode: per-block partial sums
  int *err;            // latched error word
  StepParams p;
  ConstT<T> c;
  // per-direction plane pointers (kernel parameters: one address op per access)
  const S *fin[QMAX], *gin[QMAX];
  S *fout[QMAX], *gout[QMAX];
  // g held as g_eq (tau_g = 1): planes A = mu - 3/2 C u.u, u_x, u_y, u_z
  T *Mp[4];
  // single-pass step: padded quads (A, C, u_x, u_y) and u_z written by the
  // step, and the padded plane sizes
  T *Qz, *Uz;
  int nxp, nyp;
};

// Error bits latched in the workspace error word.
enum : int { ERR_NONFINITE = 1, ERR_TIMEOUT = 2, ERR_BOUNDS = 4 };

// Index guard of the DSM_CHECKED build (compiled with -DDSM_CHECKED, the
// library libdsm_checked.so): every neighbour, pull, store and padded index
// the LB kernels compute passes through chk().  One outside [0, n) latches
// ERR_BOUNDS in the lattice's error word and is replaced by 0, so the access
// stays inside its buffer: the kernel reports the fault instead of making it.
// In the normal build chk() is the identity.  (Host-callable so that the
// index arithmetic can be checked on the CPU.)
template <class I>
__host__ __device__ __forceinline__ I chk(int *err, I i, long long n) {
#ifdef DSM_CHECKED
  if (i < 0 || (long long)i >= n) {
#ifdef __CUDA_ARCH__
    if (err) atomicOr(err, ERR_BOUNDS);
#else
    if (err) *err |= ERR_BOUNDS;
#endif
    return I(0);
  }
#else
  (void)err;
  (void)n;
#endif
  return i;
}

// Type-erased launch arguments: the ABI layer fills these and calls through an
// LBTable, so that each precision compiles in its own translation unit.
struct LBRaw {
  int nx, ny, nz;
  long long N, pitch;
  const void *f_in, *g_in;
  const float *g0_in;
  void *f_out, *g_out;
  float *g0_out;
  void *C;
  const void *Cprev;
  const void *C1;
  const unsigned char *mask;
  void *M;          // 4 planes of pitch reals (see LBArgs::Mp)
  void *Qz, *Uz;    // single-pass step outputs (see LBArgs::Qz)
  int nxp, nyp;
  int eq;           // the fused pass stores g as g_eq (A, u) instead of populations
  int implicit;     // the current g are held as g_eq (A, u, Cprev)
  void *out;
  int field_sel;
  double *partials;
  int *err;
  StepParams p;
};

// One lattice of a batched launch: its arguments for either current buffer.
struct BatchRaw {
  LBRaw r[2];         // r[p]: reads buffer p, writes buffer 1 - p
  long long nsteps;
  int cur0;
};

// Tensor maps of the single-pass step's staged boxes: the padded quads
// (A, C, u_x, u_y) and u_z of the state it reads, and the padded C1.
struct ZMaps {
  CUtensorMap Q, U, C1;
};

struct LBTable {
  cudaError_t (*moments)(const LBRaw &, cudaStream_t);
  cudaError_t (*node)(const LBRaw &, int stage, int mode, cudaStream_t);
  cudaError_t (*init)(const LBRaw &, const void *cfield, int stage, cudaStream_t);
  cudaError_t (*solid)(const void *sd, void *c1, long long N, double alpha_s, cudaStream_t);
  cudaError_t (*get_pops)(const LBRaw &, void *f, void *g, cudaStream_t);
  cudaError_t (*set_pops)(const LBRaw &, const void *f, const void *g, cudaStream_t);
  cudaError_t (*materialize)(const LBRaw &, cudaStream_t);  // g_eq -> populations of g_out
  cudaError_t (*batch)(const BatchRaw *items, int n, void *scratch, size_t bytes, bool rc,
                       bool eq, unsigned long long spins, cudaStream_t);
  size_t (*batch_bytes)(const BatchRaw *items, int n);
  // single-pass step (D3Q19, g held as g_eq, periodic; see dsm_zstep.cuh):
  // one step from the padded state the maps describe into r.Qz / r.Uz;
  // resident blocks per SM; canonical state <-> padded buffers
  cudaError_t (*zstep)(const LBRaw &r, const ZMaps &m, int zrun, cudaStream_t);
  int (*zresident)();
  cudaError_t (*zpack)(const LBRaw &r, void *Qz0, void *Qz1, void *Uz0, void *Uz1, void *C1z,
                       cudaStream_t);
  cudaError_t (*zunpack)(const LBRaw &r, const void *Qz, const void *Uz, void *Cout, cudaStream_t);
  int q, real_bytes, store_bytes;
  bool k16;
};

// One table per (lattice, precision); defined in dsm_lb_<precision>.cu.
LBTable lb_table_f64(int kind);
LBTable lb_table_f32(int kind);
LBTable lb_table_bf16(int kind);
LBTable lb_table_f16(int kind);

// Faces of dsm_params: each 0..2, an axis periodic on both faces or neither,
// the z faces of a D2Q9 lattice periodic.
inline bool faces_valid(const dsm_params *p) {
  for (int a = 0; a < 3; a++) {
    const int lo = p->face[2 * a], hi = p->face[2 * a + 1];
    if (lo < 0 || lo > 2 || hi < 0 || hi > 2) return false;
    if ((lo == 0) != (hi == 0)) return false;
  }
  return !(p->lattice == DSM_D2Q9 && (p->face[4] || p->face[5]));
}
inline bool has_walls(const dsm_params *p) {
  for (int f = 0; f < 6; f++)
    if (p->face[f]) return true;
  return false;
}

__host__ __device__ inline long long round_up(long long v, long long m) {
  return (v + m - 1) / m * m;
}

}  // namespace dsm
