// dsm_em.cuh -- arguments and host entry points of the energy/gradient twin and
// the L-BFGS vector kernels (implemented in dsm_em.cu).
#pragma once

#include "dsm_common.cuh"

namespace dsm {

constexpr int FE_K = 5;              // bulk, gradient, confinement, gravity, V
constexpr long long FE_MAX_BLOCKS = 152 * 4;  // energy kernel's fixed grid: four blocks per SM
constexpr int VEC_BLOCKS = 152 * 4;  // fixed reduction grid of the vector kernels

struct FEArgs {
  int nx, ny, nz, d;
  int lo[3], hi[3];  // per axis, the coordinate one step below 0 and above n - 1
  float kappa[3];
  float a2;        // alpha^2
  float beta;      // confinement strength (active = 1)
  float fg;        // gravity force density on the liquid
  float const_grad;  // constant added to dE/dC2 (pressure constraint)
  int active;      // 1: dE/dC1, 2: dE/dC2
  const float *c1, *c2;
  const unsigned char *mask;
  float *grad;
  double *partials;
};

// FEArgs for the energy of a problem: sizes, kappa, alpha, beta, and the
// neighbour of the edge nodes per axis (periodic: the far edge; mirror or
// wall: the edge node itself).  DSM_E_INVAL for invalid faces.
dsm_status fe_args_of(const dsm_params *p, const double kappa[3], int active, double fg,
                      FEArgs *a);

// Energy of N fluid components on a frozen solid (N = nf + 1, nf free fluid
// fields C_2 .. C_N stored as nf planes; C_{N+1} = 1 - C_1 - sum of them).
constexpr int FEM_MAX_NF = 3;
struct FEMArgs {
  int nx, ny, nz;
  int lo[3], hi[3];
  int nf;                          // free fluid fields, 1 .. FEM_MAX_NF
  float kappa[FEM_MAX_NF + 2];     // kappa_1, the free fluids', the dependent fluid's
  float a2;                        // alpha^2
  float const_grad[FEM_MAX_NF];    // constant added to each free gradient (pressure form)
  long long plane;                 // nodes per field plane
  const float *c1, *c;             // solid; free fluid planes
  float *grad;                     // nf planes
  double *partials;
};
// Per free fluid: pressure dP (kcs = 0) or volume constraint kcs (V - V0)^2 / 2.
struct FEMCons {
  double dP[FEM_MAX_NF], kcs[FEM_MAX_NF], V0[FEM_MAX_NF];
};
size_t fe_multi_scratch_bytes(int kind, int nx, int ny, int nz, int nf);
// FEMArgs and FEMCons of an N-fluid energy (nfluid = N): lattice, sizes, alpha
// and faces from p, kappa_1 .. kappa_{N+1} from kappa, the constraints from
// the host arrays dP, kcs, V0 (N - 1 each, or null for zeros).  DSM_E_INVAL
// for a bad size, nfluid outside 2 .. FEM_MAX_NF + 1, a fluid kappa <= 0,
// kcs < 0 or invalid faces.
dsm_status fem_args_of(const dsm_params *p, int nfluid, const double *kappa, const double *dP,
                       const double *kcs, const double *V0, FEMArgs *a, FEMCons *cons);
cudaError_t fe_multi_launch(int kind, FEMArgs a, const FEMCons &cons, double *energy,
                            double *terms, void *scratch, cudaStream_t st);

long long fe_blocks(int kind, int nx, int ny, int nz);
size_t fe_scratch_bytes(int kind, int nx, int ny, int nz);
// defer: when given, the constraint's constant is not added to the gradient;
// *defer receives its device address (null when there is none).
cudaError_t fe_launch(int kind, FEArgs a, double dP, double kcs, double V0, double *energy,
                      double *terms, void *scratch, cudaStream_t st,
                      const double **defer = nullptr);

constexpr int LINCOMB_MAX = 64;  // most vectors one dsm_vec_lincomb combines
struct LinCoef {
  float cx;
  float c[LINCOMB_MAX];
};

size_t vec_scratch_bytes(long long n);
size_t vec_dots_scratch_bytes(long long n, int nv);
cudaError_t vec_dots(long long n, int nv, const float *V, long long stride, const float *x,
                     double *out, void *scratch, cudaStream_t st);
// A trial point's gradient and slope: g += c[0] if c is given, out[0] = g.d,
// one launch (scratch: vec_scratch_bytes(n), whose counter word starts and
// ends at zero).
cudaError_t vec_trial_slope(long long n, const double *c, float *g, const float *d, double *out,
                            void *scratch, cudaStream_t st);
// the counter word of a vec_scratch_bytes scratch (behind the block partials)
inline unsigned *vec_scratch_counter(void *scratch) {
  return (unsigned *)((char *)scratch + VEC_BLOCKS * sizeof(double));
}
// out[0] = a.a, out[1] = b.b, out[2] = c.c in one pass (scratch:
// vec_dots_scratch_bytes(n, 3))
cudaError_t vec_sumsq3(long long n, const float *a, const float *b, const float *c, double *out,
                       void *scratch, cudaStream_t st);
cudaError_t vec_lincomb(long long n, int nv, const float *V, long long stride, const double *coef,
                        const float *x, double cx, float *y, cudaStream_t st);
cudaError_t vec_dot(long long n, const float *x, const float *y, double *out, const double *scale,
                    void *scratch, cudaStream_t st);
cudaError_t vec_axpy_dev(long long n, double sign, const double *a, const double *b,
                         const float *x, float *y, cudaStream_t st);
cudaError_t vec_axpby(long long n, double a, const float *x, double b, float *y, cudaStream_t st);
cudaError_t lbfgs_direction(long long n, int m, const int *order, const float *S, const float *Y,
                            const double *rho, const double *gamma, const float *g, float *r,
                            double *alpha, void *scratch, cudaStream_t st);

}  // namespace dsm
