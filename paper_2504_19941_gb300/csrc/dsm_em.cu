// dsm_em.cu -- free energy + gradient kernel of the phase-field energy
// minimisation (Sec. II.A of the paper) and the FP64-accumulating vector
// kernels of its L-BFGS driver.
#include <math.h>
#include <string.h>

#include "dsm_em.cuh"
#include "dsm_reduce.cuh"

namespace dsm {

template <class T>
__device__ __forceinline__ T bw(T c) {
  return c * (T(1) - c) * (T(1) - T(2) * c);
}

// ---------------------------------------------------------------------------
// K4: per-node energy density and gradient (FP32), per-block FP64 partials.
//   bulk     sum_n kappa_n/2 C_n^2 (1 - C_n)^2                Eq. [frozen:bulk_energy]
//   gradient sum_n a^2 kappa_n/(2 c_s^2) sum_i w_i (C_n(x+c_i) - C_n(x))^2
//            (lattice-weighted |grad C_n|^2 of Eq. [frozen:interface_energy];
//            its exact derivative is -a^2 kappa_n L[C_n])
//   confine  beta (C1 - 1/2)^2 chi                            Eq. [frozen:poly-quadratic]
//   gravity  fg C2 h                                          Eq. [frozen:gravitational energy]
// dE/dC2 = d2 - d3 (+ constraint + fg h),  dE/dC1 = d1 - d3 + 2 beta (C1 - 1/2) chi,
// d_n = kappa_n b(C_n) - a^2 kappa_n L[C_n],  C3 = 1 - C1 - C2.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256) fe_kernel(FEArgs a, int gx, int gy, int nbricks) {
  using L = Lat<K>;
  constexpr int Q = L::Q;
  FF acc[FE_K];
#pragma unroll
  for (int k = 0; k < FE_K; k++) acc[k] = FF{0.0f, 0.0f};
  // resident blocks walk the node bricks (blockDim-shaped boxes) in a fixed
  // grid-stride order, so each block leaves one partial sum; the brick
  // coordinates advance by the stride's own (x, y, z) digits with carries
  // instead of three divisions per brick
  const int G = gridDim.x;
  const int sx = G % gx, sy = (G / gx) % gy, sz = G / (gx * gy);
  int bx = blockIdx.x % gx, by = (blockIdx.x / gx) % gy, bz = blockIdx.x / (gx * gy);
  for (int b = blockIdx.x; b < nbricks; b += G) {
    if (b != blockIdx.x) {
      bx += sx;
      by += sy;
      bz += sz;
      if (bx >= gx) {
        bx -= gx;
        by++;
      }
      if (by >= gy) {
        by -= gy;
        bz++;
      }
    }
    const int x = bx * blockDim.x + threadIdx.x;
    const int y = by * blockDim.y + threadIdx.y;
    const int z = bz * blockDim.z + threadIdx.z;
    if (!(x < a.nx && y < a.ny && z < a.nz)) continue;
    const int xm = x == 0 ? a.lo[0] : x - 1, xp = x + 1 == a.nx ? a.hi[0] : x + 1;
    const int ym = y == 0 ? a.lo[1] : y - 1, yp = y + 1 == a.ny ? a.hi[1] : y + 1;
    const int zm = z == 0 ? a.lo[2] : z - 1, zp = z + 1 == a.nz ? a.hi[2] : z + 1;
    const int s = a.nx * a.ny;
    const int ox[3] = {xm, x, xp}, oy[3] = {ym * a.nx, y * a.nx, yp * a.nx},
              oz[3] = {zm * s, z * s, zp * s};
    const int n = x + y * a.nx + z * s;
    const float k1 = a.kappa[0], k2 = a.kappa[1], k3 = a.kappa[2];
    const float c1 = a.c1[n], c2 = a.c2[n], c3 = 1.0f - c1 - c2;
    // C3 = 1 - C1 - C2, so its differences are -(d1 + d2): L[C3] = -L[C1] - L[C2]
    // and its pair sum is p1 + p2 + 2 x12 with x12 = sum_i w_i d1 d2
    float l1 = 0.f, l2 = 0.f, p1 = 0.f, p2 = 0.f, x12 = 0.f;
#pragma unroll
    for (int i = 1; i < Q; i++) {
      const int m = ox[L::cx(i) + 1] + oy[L::cy(i) + 1] + oz[L::cz(i) + 1];
      const float w = float(L::w(i));
      const float d1 = __ldg(a.c1 + m) - c1, d2 = __ldg(a.c2 + m) - c2;
      const float t1 = w * d1, t2 = w * d2;
      l1 += t1;
      l2 += t2;
      p1 = fmaf(t1, d1, p1);
      p2 = fmaf(t2, d2, p2);
      x12 = fmaf(t1, d2, x12);
    }
    const float p3 = p1 + p2 + 2.0f * x12;
    l1 *= 6.f;
    l2 *= 6.f;
    const float l3 = -(l1 + l2);
    const float A2 = a.a2;
    // per-node densities in FP32, accumulated with carried rounding errors
    const float q1 = c1 * (1.0f - c1), q2 = c2 * (1.0f - c2), q3 = c3 * (1.0f - c3);
    acc[0] = ff_add(acc[0], FF{0.5f * (k1 * q1 * q1 + k2 * q2 * q2 + k3 * q3 * q3), 0.0f});
    acc[1] = ff_add(acc[1], FF{1.5f * A2 * (k1 * p1 + k2 * p2 + k3 * p3), 0.0f});
    const bool inS = a.mask ? a.mask[n] != 0 : false;
    const bool chi = (inS && c1 < 0.5f) || (!inS && c1 > 0.5f);
    if (a.active == 1 && chi) acc[2] = ff_add(acc[2], FF{a.beta * (c1 - 0.5f) * (c1 - 0.5f), 0.0f});
    const int hgt = (a.d == 2) ? y : z;
    acc[3] = ff_add(acc[3], FF{a.fg * c2 * (float)hgt, 0.0f});
    acc[4] = ff_add(acc[4], FF{c2, 0.0f});
    const float dd1 = k1 * bw(c1) - A2 * k1 * l1;
    const float dd2 = k2 * bw(c2) - A2 * k2 * l2;
    const float dd3 = k3 * bw(c3) - A2 * k3 * l3;
    float gr;
    if (a.active == 2) gr = dd2 - dd3 + a.const_grad + a.fg * (float)hgt;
    else gr = dd1 - dd3 + (chi ? 2.0f * a.beta * (c1 - 0.5f) : 0.0f);
    a.grad[n] = gr;
  }
  const int sums[FE_K] = {0, 0, 0, 0, 0};
  block_reduce_ff<FE_K>(acc, sums, a.partials + (long long)blockIdx.x * FE_K);
}

// Sum the per-block partials in block order; assemble E and the constraint.
__global__ void fe_finalize_kernel(const double *partials, long long nb, double dP, double kcs,
                                   double V0, double *energy, double *terms, double *dEcs) {
  __shared__ double sh[FE_K][256];
  double s[FE_K] = {0, 0, 0, 0, 0};
  for (long long b = threadIdx.x; b < nb; b += blockDim.x)
    for (int k = 0; k < FE_K; k++) s[k] += partials[b * FE_K + k];
  for (int k = 0; k < FE_K; k++) sh[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int k = 0; k < FE_K; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double V = sh[4][0];
    const double Ecs = (kcs == 0.0) ? -dP * V : 0.5 * kcs * (V - V0) * (V - V0);
    const double E = sh[0][0] + sh[1][0] + sh[2][0] + Ecs + sh[3][0];
    if (energy) energy[0] = E;
    if (terms) {
      terms[0] = sh[0][0];
      terms[1] = sh[1][0];
      terms[2] = sh[2][0];
      terms[3] = Ecs;
      terms[4] = sh[3][0];
      terms[5] = V;
    }
    dEcs[0] = (kcs == 0.0) ? -dP : kcs * (V - V0);
  }
}

__global__ void add_dev_scalar_kernel(long long n, const double *c, float *g) {
  const float v = (float)c[0];
  const long long G = (long long)gridDim.x * blockDim.x;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; k + 3 * G < n; k += 4 * G) {  // four loads in flight per thread
    const float a0 = g[k], a1 = g[k + G], a2 = g[k + 2 * G], a3 = g[k + 3 * G];
    g[k] = a0 + v;
    g[k + G] = a1 + v;
    g[k + 2 * G] = a2 + v;
    g[k + 3 * G] = a3 + v;
  }
  for (; k < n; k += G) g[k] += v;
}

dsm_status fem_args_of(const dsm_params *p, int nfluid, const double *kappa, const double *dP,
                       const double *kcs, const double *V0, FEMArgs *a, FEMCons *cons) {
  if (!p || !kappa || !a || !cons) return DSM_E_INVAL;
  if (p->lattice != DSM_D2Q9 && p->lattice != DSM_D3Q19) return DSM_E_INVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->lattice == DSM_D2Q9 && p->nz != 1))
    return DSM_E_INVAL;
  if ((long long)p->nx * p->ny * p->nz >= (1ll << 31)) return DSM_E_INVAL;
  if (nfluid < 2 || nfluid > FEM_MAX_NF + 1 || !(p->alpha > 0.0)) return DSM_E_INVAL;
  if (!faces_valid(p)) return DSM_E_INVAL;
  memset(a, 0, sizeof(*a));
  memset(cons, 0, sizeof(*cons));
  a->nx = p->nx;
  a->ny = p->ny;
  a->nz = p->nz;
  const int n[3] = {p->nx, p->ny, p->nz};
  for (int i = 0; i < 3; i++) {
    a->lo[i] = p->face[2 * i] ? 0 : n[i] - 1;
    a->hi[i] = p->face[2 * i + 1] ? n[i] - 1 : 0;
  }
  a->nf = nfluid - 1;
  for (int k = 0; k <= nfluid; k++) {
    if (k > 0 && !(kappa[k] > 0.0)) return DSM_E_INVAL;  // every fluid needs its bulk term
    if (!isfinite(kappa[k])) return DSM_E_INVAL;
    a->kappa[k] = (float)kappa[k];
  }
  for (int f = 0; f < a->nf; f++) {
    cons->dP[f] = dP ? dP[f] : 0.0;
    cons->kcs[f] = kcs ? kcs[f] : 0.0;
    cons->V0[f] = V0 ? V0[f] : 0.0;
    if (cons->kcs[f] < 0.0) return DSM_E_INVAL;
  }
  a->a2 = (float)(p->alpha * p->alpha);
  a->plane = (long long)p->nx * p->ny * p->nz;
  return DSM_OK;
}

dsm_status fe_args_of(const dsm_params *p, const double kappa[3], int active, double fg,
                      FEArgs *a) {
  memset(a, 0, sizeof(*a));
  a->nx = p->nx;
  a->ny = p->ny;
  a->nz = p->nz;
  a->d = p->lattice == DSM_D2Q9 ? 2 : 3;
  if (!faces_valid(p)) return DSM_E_INVAL;
  const int n[3] = {p->nx, p->ny, p->nz};
  for (int i = 0; i < 3; i++) {
    // a mirror or wall plane half a node outside the edge maps the step back
    // onto the edge node: the lattice is half of a mirror-symmetric periodic one
    a->lo[i] = p->face[2 * i] ? 0 : n[i] - 1;
    a->hi[i] = p->face[2 * i + 1] ? n[i] - 1 : 0;
    a->kappa[i] = (float)kappa[i];
  }
  a->a2 = (float)(p->alpha * p->alpha);
  a->beta = (float)p->beta;
  a->fg = (float)fg;
  a->active = active;
  return DSM_OK;
}

static dim3 fe_block(int kind) { return kind == 0 ? dim3(32, 8, 1) : dim3(32, 4, 2); }
static dim3 fe_bricks(int kind, int nx, int ny, int nz) {
  const dim3 b = fe_block(kind);
  return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y, (nz + b.z - 1) / b.z);
}

// blocks (= partial sums) of one evaluation
long long fe_blocks(int kind, int nx, int ny, int nz) {
  const dim3 g = fe_bricks(kind, nx, ny, nz);
  const long long nb = (long long)g.x * g.y * g.z;
  return nb < FE_MAX_BLOCKS ? nb : FE_MAX_BLOCKS;
}

size_t fe_scratch_bytes(int kind, int nx, int ny, int nz) {
  return (size_t)round_up(fe_blocks(kind, nx, ny, nz) * FE_K * sizeof(double), 256) + 256;
}

cudaError_t fe_launch(int kind, FEArgs a, double dP, double kcs, double V0, double *energy,
                      double *terms, void *scratch, cudaStream_t st, const double **defer) {
  const long long nb = fe_blocks(kind, a.nx, a.ny, a.nz);
  double *partials = (double *)scratch;
  double *dEcs = (double *)((char *)scratch + round_up(nb * FE_K * sizeof(double), 256));
  a.partials = partials;
  a.const_grad = (kcs == 0.0) ? (float)(-dP) : 0.0f;
  const dim3 g = fe_bricks(kind, a.nx, a.ny, a.nz);
  const int nbricks = (int)((long long)g.x * g.y * g.z);
  if (kind == 0) fe_kernel<0><<<(unsigned)nb, fe_block(0), 0, st>>>(a, g.x, g.y, nbricks);
  else fe_kernel<1><<<(unsigned)nb, fe_block(1), 0, st>>>(a, g.x, g.y, nbricks);
  fe_finalize_kernel<<<1, 256, 0, st>>>(partials, nb, dP, kcs, V0, energy, terms, dEcs);
  if (defer) {  // the caller adds the constraint's constant (null: none)
    *defer = (kcs != 0.0 && a.active == 2) ? dEcs : nullptr;
    return cudaGetLastError();
  }
  if (kcs != 0.0 && a.active == 2) {
    const long long N = (long long)a.nx * a.ny * a.nz;
    long long blocks = (N + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    add_dev_scalar_kernel<<<(int)blocks, 256, 0, st>>>(N, dEcs, a.grad);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K4 for N fluid components (N = NF + 1 fluids, NF free fields): the same
// per-component terms with C_{N+1} = 1 - C_1 - sum_f C_f, whose differences are
// minus the sum of the others'.  dE/dC_f = d_f - d_{N+1} (+ the constraint),
// d_k = kappa_k b(C_k) - a^2 kappa_k L[C_k].  Per-block FP64 partials: bulk,
// gradient, then V_f of each free fluid.
// ---------------------------------------------------------------------------
template <int K, int NF>
__global__ void __launch_bounds__(256) fe_multi_kernel(FEMArgs a, int gx, int gy, int nbricks) {
  using L = Lat<K>;
  constexpr int Q = L::Q;
  constexpr int NC = NF + 2;  // components: solid, free fluids, dependent fluid
  constexpr int NA = 2 + NF;
  FF acc[NA];
#pragma unroll
  for (int k = 0; k < NA; k++) acc[k] = FF{0.0f, 0.0f};
  const int G = gridDim.x;
  const int sx = G % gx, sy = (G / gx) % gy, sz = G / (gx * gy);
  int bx = blockIdx.x % gx, by = (blockIdx.x / gx) % gy, bz = blockIdx.x / (gx * gy);
  for (int b = blockIdx.x; b < nbricks; b += G) {
    if (b != blockIdx.x) {
      bx += sx;
      by += sy;
      bz += sz;
      if (bx >= gx) {
        bx -= gx;
        by++;
      }
      if (by >= gy) {
        by -= gy;
        bz++;
      }
    }
    const int x = bx * blockDim.x + threadIdx.x;
    const int y = by * blockDim.y + threadIdx.y;
    const int z = bz * blockDim.z + threadIdx.z;
    if (!(x < a.nx && y < a.ny && z < a.nz)) continue;
    const int xm = x == 0 ? a.lo[0] : x - 1, xp = x + 1 == a.nx ? a.hi[0] : x + 1;
    const int ym = y == 0 ? a.lo[1] : y - 1, yp = y + 1 == a.ny ? a.hi[1] : y + 1;
    const int zm = z == 0 ? a.lo[2] : z - 1, zp = z + 1 == a.nz ? a.hi[2] : z + 1;
    const int s = a.nx * a.ny;
    const int ox[3] = {xm, x, xp}, oy[3] = {ym * a.nx, y * a.nx, yp * a.nx},
              oz[3] = {zm * s, z * s, zp * s};
    const int n = x + y * a.nx + z * s;
    float cv[NC];
    cv[0] = a.c1[n];
    float last = 1.0f - cv[0];
#pragma unroll
    for (int f = 0; f < NF; f++) {
      cv[1 + f] = a.c[f * a.plane + n];
      last -= cv[1 + f];
    }
    cv[NC - 1] = last;
    float l[NC], p[NC];
#pragma unroll
    for (int k = 0; k < NC; k++) l[k] = p[k] = 0.0f;
#pragma unroll
    for (int i = 1; i < Q; i++) {
      const int m = ox[L::cx(i) + 1] + oy[L::cy(i) + 1] + oz[L::cz(i) + 1];
      const float w = float(L::w(i));
      float dsum = 0.0f;
#pragma unroll
      for (int k = 0; k < NC - 1; k++) {
        const float v = k == 0 ? __ldg(a.c1 + m) : __ldg(a.c + (k - 1) * a.plane + m);
        const float d = v - cv[k];
        const float t = w * d;
        l[k] += t;
        p[k] = fmaf(t, d, p[k]);
        dsum += d;
      }
      // the dependent fluid's difference is -dsum
      l[NC - 1] -= w * dsum;
      p[NC - 1] = fmaf(w * dsum, dsum, p[NC - 1]);
    }
    float bulk = 0.0f, grd = 0.0f, dd[NC];
#pragma unroll
    for (int k = 0; k < NC; k++) {
      const float q = cv[k] * (1.0f - cv[k]);
      bulk += 0.5f * a.kappa[k] * q * q;
      grd += a.kappa[k] * p[k];
      dd[k] = a.kappa[k] * bw(cv[k]) - a.a2 * a.kappa[k] * (6.0f * l[k]);
    }
    acc[0] = ff_add(acc[0], FF{bulk, 0.0f});
    acc[1] = ff_add(acc[1], FF{1.5f * a.a2 * grd, 0.0f});
#pragma unroll
    for (int f = 0; f < NF; f++) {
      acc[2 + f] = ff_add(acc[2 + f], FF{cv[1 + f], 0.0f});
      a.grad[f * a.plane + n] = dd[1 + f] - dd[NC - 1] + a.const_grad[f];
    }
  }
  int sums[NA];
#pragma unroll
  for (int k = 0; k < NA; k++) sums[k] = 0;
  block_reduce_ff<NA>(acc, sums, a.partials + (long long)blockIdx.x * NA);
}

// Sum the per-block partials in block order; assemble E, the terms (bulk,
// gradient, constraint, V_f) and each free fluid's constraint derivative.
template <int NF>
__global__ void fe_multi_finalize_kernel(const double *partials, long long nb, FEMCons cons,
                                         double *energy, double *terms, double *dEcs) {
  constexpr int NA = 2 + NF;
  __shared__ double sh[NA][256];
  double s[NA];
  for (int k = 0; k < NA; k++) s[k] = 0.0;
  for (long long b = threadIdx.x; b < nb; b += blockDim.x)
    for (int k = 0; k < NA; k++) s[k] += partials[b * NA + k];
  for (int k = 0; k < NA; k++) sh[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int k = 0; k < NA; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double Ecs = 0.0;
    for (int f = 0; f < NF; f++) {
      const double V = sh[2 + f][0];
      const bool press = cons.kcs[f] == 0.0;
      Ecs += press ? -cons.dP[f] * V : 0.5 * cons.kcs[f] * (V - cons.V0[f]) * (V - cons.V0[f]);
      dEcs[f] = press ? -cons.dP[f] : cons.kcs[f] * (V - cons.V0[f]);
      if (terms) terms[3 + f] = V;
    }
    const double E = sh[0][0] + sh[1][0] + Ecs;
    if (energy) energy[0] = E;
    if (terms) {
      terms[0] = sh[0][0];
      terms[1] = sh[1][0];
      terms[2] = Ecs;
    }
  }
}

size_t fe_multi_scratch_bytes(int kind, int nx, int ny, int nz, int nf) {
  return (size_t)round_up(fe_blocks(kind, nx, ny, nz) * (2 + nf) * sizeof(double), 256) + 256;
}

template <int K, int NF>
static cudaError_t fe_multi_run(FEMArgs a, const FEMCons &cons, double *energy, double *terms,
                                void *scratch, cudaStream_t st) {
  const long long nb = fe_blocks(K, a.nx, a.ny, a.nz);
  double *partials = (double *)scratch;
  double *dEcs = (double *)((char *)scratch + round_up(nb * (2 + NF) * sizeof(double), 256));
  a.partials = partials;
  for (int f = 0; f < NF; f++) a.const_grad[f] = cons.kcs[f] == 0.0 ? (float)(-cons.dP[f]) : 0.0f;
  const dim3 g = fe_bricks(K, a.nx, a.ny, a.nz);
  const int nbricks = (int)((long long)g.x * g.y * g.z);
  fe_multi_kernel<K, NF><<<(unsigned)nb, fe_block(K), 0, st>>>(a, g.x, g.y, nbricks);
  fe_multi_finalize_kernel<NF><<<1, 256, 0, st>>>(partials, nb, cons, energy, terms, dEcs);
  const long long N = (long long)a.nx * a.ny * a.nz;
  long long blocks = (N + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  for (int f = 0; f < NF; f++)
    if (cons.kcs[f] != 0.0)
      add_dev_scalar_kernel<<<(int)blocks, 256, 0, st>>>(N, dEcs + f, a.grad + f * a.plane);
  return cudaGetLastError();
}

cudaError_t fe_multi_launch(int kind, FEMArgs a, const FEMCons &cons, double *energy,
                            double *terms, void *scratch, cudaStream_t st) {
  switch (kind * 4 + a.nf) {
    case 1: return fe_multi_run<0, 1>(a, cons, energy, terms, scratch, st);
    case 2: return fe_multi_run<0, 2>(a, cons, energy, terms, scratch, st);
    case 3: return fe_multi_run<0, 3>(a, cons, energy, terms, scratch, st);
    case 5: return fe_multi_run<1, 1>(a, cons, energy, terms, scratch, st);
    case 6: return fe_multi_run<1, 2>(a, cons, energy, terms, scratch, st);
    case 7: return fe_multi_run<1, 3>(a, cons, energy, terms, scratch, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// K6: L-BFGS vector kernels.  Fixed grid (VEC_BLOCKS x 256), grid-stride in a
// fixed order, FP64 accumulation, block partials summed in block order: the
// result does not depend on timing.  Every grid-stride loop takes four
// elements a grid apart per iteration, so that four loads per stream are in
// flight (the order of the elements, and so of every sum, is unchanged).
// ---------------------------------------------------------------------------

static int vec_grid(long long n);

// The exact product a b (TwoProd: p + e, e from one FMA) added to the pair s:
// TwoSum into s.hi, both rounding errors into s.lo.  FP64 accuracy from FP32
// instructions, without renormalising the pair at every element.
__device__ __forceinline__ void acc_prod(FF &s, float a, float b) {
  const float p = a * b;
  const float pe = fmaf(a, b, -p);
  const FF t = two_sum(s.hi, p);
  s.hi = t.hi;
  s.lo += t.lo + pe;
}

// The last block of a grid sums the grid's partials in block order (as
// dot_finalize_kernel does) into out[0] and rearms the counter: each block
// publishes its partial, counts itself, and the block that counts last (every
// other partial is then visible) finishes.  No block waits for another.
__device__ __forceinline__ void last_block_sum(const double *partials, unsigned *counter,
                                               double *out) {
  __shared__ bool last;
  __shared__ double sh[256];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
    s += ((volatile const double *)partials)[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sh[0];
    *counter = 0u;
  }
}

// A trial point's gradient completed and its slope: g += c[0] (the
// constraint's constant, when c is given), out[0] = g.d, in one pass (the
// sum as dot_kernel's); blockDim.x = 256.
__global__ void __launch_bounds__(256) trial_slope_kernel(long long n, const double *c, float *g,
                                                          const float *d, double *partials,
                                                          unsigned *counter, double *out) {
  const float cv = c ? (float)c[0] : 0.0f;
  FF s[1] = {FF{0.0f, 0.0f}};
  const long long G = (long long)gridDim.x * blockDim.x;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; k + 3 * G < n; k += 4 * G) {
    float gg[4], dd[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      gg[u] = g[k + u * G];
      dd[u] = d[k + u * G];
    }
    if (c) {
#pragma unroll
      for (int u = 0; u < 4; u++) {
        gg[u] += cv;
        g[k + u * G] = gg[u];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; u++) acc_prod(s[0], gg[u], dd[u]);
  }
  for (; k < n; k += G) {
    float gk = g[k];
    if (c) {
      gk += cv;
      g[k] = gk;
    }
    acc_prod(s[0], gk, d[k]);
  }
  const int sums[1] = {0};
  block_reduce_ff<1>(s, sums, partials + blockIdx.x);
  last_block_sum(partials, counter, out);
}

cudaError_t vec_trial_slope(long long n, const double *c, float *g, const float *d, double *out,
                            void *scratch, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  double *partials = (double *)scratch;
  unsigned *counter = vec_scratch_counter(scratch);
  trial_slope_kernel<<<vec_grid(n), 256, 0, st>>>(n, c, g, d, partials, counter, out);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) dot_kernel(long long n, const float *x, const float *y,
                                                  double *partials) {
  FF s[1] = {FF{0.0f, 0.0f}};
  const long long G = (long long)gridDim.x * blockDim.x;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; k + 3 * G < n; k += 4 * G) {
    const float x0 = x[k], x1 = x[k + G], x2 = x[k + 2 * G], x3 = x[k + 3 * G];
    const float y0 = y[k], y1 = y[k + G], y2 = y[k + 2 * G], y3 = y[k + 3 * G];
    acc_prod(s[0], x0, y0);
    acc_prod(s[0], x1, y1);
    acc_prod(s[0], x2, y2);
    acc_prod(s[0], x3, y3);
  }
  for (; k < n; k += G) acc_prod(s[0], x[k], y[k]);
  const int sums[1] = {0};
  block_reduce_ff<1>(s, sums, partials + blockIdx.x);
}

__global__ void dot_finalize_kernel(const double *partials, int nb, const double *scale,
                                    double *out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partials[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = (scale ? scale[0] : 1.0) * sh[0];
}

// Batched dot products V_k . x for k < nv (V_k at V + k * stride): one launch,
// grid (blocks, nv); the same fixed grid-stride order and carried-error sums as
// dot_kernel, so each result equals a separate vec_dot of the same vectors.
__global__ void __launch_bounds__(256) dots_kernel(long long n, const float *V, long long stride,
                                                   const float *x, double *partials) {
  const float *v = V + blockIdx.y * stride;
  FF s[1] = {FF{0.0f, 0.0f}};
  const long long G = (long long)gridDim.x * blockDim.x;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; k + 3 * G < n; k += 4 * G) {
    const float v0 = v[k], v1 = v[k + G], v2 = v[k + 2 * G], v3 = v[k + 3 * G];
    const float x0 = x[k], x1 = x[k + G], x2 = x[k + 2 * G], x3 = x[k + 3 * G];
    acc_prod(s[0], v0, x0);
    acc_prod(s[0], v1, x1);
    acc_prod(s[0], v2, x2);
    acc_prod(s[0], v3, x3);
  }
  for (; k < n; k += G) acc_prod(s[0], v[k], x[k]);
  const int sums[1] = {0};
  block_reduce_ff<1>(s, sums, partials + (long long)blockIdx.y * gridDim.x + blockIdx.x);
}

// a.a, b.b and c.c in one pass: partials (block) hold the three sums side by
// side; each sum as dot_kernel's
__global__ void __launch_bounds__(256) sumsq3_kernel(long long n, const float *a, const float *b,
                                                     const float *c, double *partials) {
  FF s[3] = {FF{0.0f, 0.0f}, FF{0.0f, 0.0f}, FF{0.0f, 0.0f}};
  const long long G = (long long)gridDim.x * blockDim.x;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; k + 3 * G < n; k += 4 * G) {
    float aa[4], bb[4], cc[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      aa[u] = a[k + u * G];
      bb[u] = b[k + u * G];
      cc[u] = c[k + u * G];
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      acc_prod(s[0], aa[u], aa[u]);
      acc_prod(s[1], bb[u], bb[u]);
      acc_prod(s[2], cc[u], cc[u]);
    }
  }
  for (; k < n; k += G) {
    const float ak = a[k], bk = b[k], ck = c[k];
    acc_prod(s[0], ak, ak);
    acc_prod(s[1], bk, bk);
    acc_prod(s[2], ck, ck);
  }
  const int sums[3] = {0, 0, 0};
  block_reduce_ff<3>(s, sums, partials + 3 * (long long)blockIdx.x);
}

// block t: partial t of every block (partials[stride b + t]) summed in block order
__global__ void strided_finalize_kernel(const double *partials, int nb, int stride, double *out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partials[(long long)stride * b + blockIdx.x];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// one block per dot product: its block partials summed in block order
__global__ void dots_finalize_kernel(const double *partials, int nb, double *out) {
  __shared__ double sh[256];
  const double *p = partials + (long long)blockIdx.x * nb;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += p[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// y = cx x + sum_k c_k V_k, coefficients passed by value, the sum in k order
__global__ void __launch_bounds__(256) lincomb_kernel(long long n, int nv, const float *V,
                                                      long long stride, LinCoef c,
                                                      const float *x, float *y) {
  const long long G = (long long)gridDim.x * blockDim.x;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; k + 3 * G < n; k += 4 * G) {
    float acc[4];
#pragma unroll
    for (int u = 0; u < 4; u++) acc[u] = c.cx * x[k + u * G];
    for (int j = 0; j < nv; j++) {
      const float *vj = V + j * stride + k;
      float vv[4];
#pragma unroll
      for (int u = 0; u < 4; u++) vv[u] = vj[u * G];
#pragma unroll
      for (int u = 0; u < 4; u++) acc[u] += c.c[j] * vv[u];
    }
#pragma unroll
    for (int u = 0; u < 4; u++) y[k + u * G] = acc[u];
  }
  for (; k < n; k += G) {
    float acc = c.cx * x[k];
    for (int j = 0; j < nv; j++) acc += c.c[j] * V[j * stride + k];
    y[k] = acc;
  }
}

// y += sign * (a[0] - (b ? b[0] : 0)) * x
__global__ void __launch_bounds__(256) axpy_dev_kernel(long long n, double sign, const double *a,
                                                       const double *b, const float *x, float *y) {
  const float c = (float)(sign * (a[0] - (b ? b[0] : 0.0)));
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    y[k] += c * x[k];
}

__global__ void __launch_bounds__(256) axpby_kernel(long long n, float a, const float *x, float b,
                                                    float *y) {
  const long long G = (long long)gridDim.x * blockDim.x;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b == 0.0f) {
    for (; k + 3 * G < n; k += 4 * G) {
      const float x0 = x[k], x1 = x[k + G], x2 = x[k + 2 * G], x3 = x[k + 3 * G];
      y[k] = a * x0;
      y[k + G] = a * x1;
      y[k + 2 * G] = a * x2;
      y[k + 3 * G] = a * x3;
    }
    for (; k < n; k += G) y[k] = a * x[k];
  } else {
    for (; k < n; k += G) y[k] = a * x[k] + b * y[k];
  }
}

// y = s[0] * x
__global__ void __launch_bounds__(256) scale_dev_kernel(long long n, const double *s, const float *x,
                                                        float *y) {
  const float c = (float)s[0];
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    y[k] = c * x[k];
}

static int vec_grid(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < VEC_BLOCKS ? (b > 0 ? b : 1) : VEC_BLOCKS);
}

size_t vec_scratch_bytes(long long) { return VEC_BLOCKS * sizeof(double) + 256; }

size_t vec_dots_scratch_bytes(long long n, int nv) {
  return (size_t)(nv > 0 ? nv : 1) * vec_grid(n) * sizeof(double) + 256;
}

cudaError_t vec_sumsq3(long long n, const float *a, const float *b, const float *c, double *out,
                       void *scratch, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int g = vec_grid(n);
  double *partials = (double *)scratch;
  sumsq3_kernel<<<g, 256, 0, st>>>(n, a, b, c, partials);
  strided_finalize_kernel<<<3, 256, 0, st>>>(partials, g, 3, out);
  return cudaGetLastError();
}

cudaError_t vec_dots(long long n, int nv, const float *V, long long stride, const float *x,
                     double *out, void *scratch, cudaStream_t st) {
  if (nv <= 0) return cudaSuccess;
  double *partials = (double *)scratch;
  const int g = vec_grid(n);
  dots_kernel<<<dim3(g, nv), 256, 0, st>>>(n, V, stride, x, partials);
  dots_finalize_kernel<<<nv, 256, 0, st>>>(partials, g, out);
  return cudaGetLastError();
}

cudaError_t vec_lincomb(long long n, int nv, const float *V, long long stride, const double *coef,
                        const float *x, double cx, float *y, cudaStream_t st) {
  LinCoef c;
  c.cx = (float)cx;
  for (int j = 0; j < LINCOMB_MAX; j++) c.c[j] = j < nv ? (float)coef[j] : 0.0f;
  lincomb_kernel<<<vec_grid(n), 256, 0, st>>>(n, nv, V, stride, c, x, y);
  return cudaGetLastError();
}

cudaError_t vec_dot(long long n, const float *x, const float *y, double *out, const double *scale,
                    void *scratch, cudaStream_t st) {
  double *partials = (double *)scratch;
  const int g = vec_grid(n);
  dot_kernel<<<g, 256, 0, st>>>(n, x, y, partials);
  dot_finalize_kernel<<<1, 256, 0, st>>>(partials, g, scale, out);
  return cudaGetLastError();
}

cudaError_t vec_axpy_dev(long long n, double sign, const double *a, const double *b,
                         const float *x, float *y, cudaStream_t st) {
  axpy_dev_kernel<<<vec_grid(n), 256, 0, st>>>(n, sign, a, b, x, y);
  return cudaGetLastError();
}

cudaError_t vec_axpby(long long n, double a, const float *x, double b, float *y, cudaStream_t st) {
  axpby_kernel<<<vec_grid(n), 256, 0, st>>>(n, (float)a, x, (float)b, y);
  return cudaGetLastError();
}

// Two-loop recursion (Nocedal & Wright Algorithm 7.4): r = -H g.
cudaError_t lbfgs_direction(long long n, int m, const int *order, const float *S, const float *Y,
                            const double *rho, const double *gamma, const float *g, float *r,
                            double *alpha, void *scratch, cudaStream_t st) {
  double *beta = (double *)((char *)scratch + VEC_BLOCKS * sizeof(double));
  cudaError_t e;
  // q = g (held in r)
  axpby_kernel<<<vec_grid(n), 256, 0, st>>>(n, 1.0f, g, 0.0f, r);
  for (int k = m - 1; k >= 0; k--) {  // newest to oldest
    const long long s = order[k];
    if ((e = vec_dot(n, S + s * n, r, alpha + k, rho + s, scratch, st)) != cudaSuccess) return e;
    axpy_dev_kernel<<<vec_grid(n), 256, 0, st>>>(n, -1.0, alpha + k, nullptr, Y + s * n, r);
  }
  scale_dev_kernel<<<vec_grid(n), 256, 0, st>>>(n, gamma, r, r);
  for (int k = 0; k < m; k++) {  // oldest to newest
    const long long s = order[k];
    if ((e = vec_dot(n, Y + s * n, r, beta, rho + s, scratch, st)) != cudaSuccess) return e;
    axpy_dev_kernel<<<vec_grid(n), 256, 0, st>>>(n, 1.0, alpha + k, beta, S + s * n, r);
  }
  axpby_kernel<<<vec_grid(n), 256, 0, st>>>(n, -1.0f, r, 0.0f, r);
  return cudaGetLastError();
}

}  // namespace dsm
