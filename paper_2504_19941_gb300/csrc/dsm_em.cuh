// dsm_em.cuh -- arguments and host entry points of the energy/gradient twin and
// the L-BFGS vector kernels (implemented in dsm_em.cu).
#pragma once

#include "dsm_common.cuh"

namespace dsm {

constexpr int FE_K = 5;              // bulk, gradient, confinement, gravity, V
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

long long fe_blocks(int kind, int nx, int ny, int nz);
size_t fe_scratch_bytes(int kind, int nx, int ny, int nz);
cudaError_t fe_launch(int kind, FEArgs a, double dP, double kcs, double V0, double *energy,
                      double *terms, void *scratch, cudaStream_t st);

constexpr int LINCOMB_MAX = 64;  // most vectors one dsm_vec_lincomb combines
struct LinCoef {
  float cx;
  float c[LINCOMB_MAX];
};

size_t vec_scratch_bytes(long long n);
size_t vec_dots_scratch_bytes(long long n, int nv);
cudaError_t vec_dots(long long n, int nv, const float *V, long long stride, const float *x,
                     double *out, void *scratch, cudaStream_t st);
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
