// dsm_noalloc.cu -- dsm_fe_energy_grad_noalloc: the free-energy/gradient entry
// point for callers that cannot allocate device memory at all.
//
// dsm_fe_energy_grad asks its caller for a scratch buffer.  Some callers have
// no way to provide one: a host program that links only this library and has no
// CUDA allocator of its own to call, or an application whose device memory is
// entirely owned by another allocator that forbids side allocations.  This
// variant takes its scratch from a fixed array that lives in the library's own
// device image instead, so the caller passes only inputs and outputs.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (DSM_NOALLOC_SCRATCH_BYTES) until the process exits.  All
// calls on a device share it, so two calls whose kernels overlap on the GPU
// race on it.  Nothing in it has to start at zero: every word a call reads was
// written earlier in the same call (block partial sums, then the constraint
// term).
#include <string.h>

#include "dsm_em.cuh"
#include "dsm_trace.cuh"

using namespace dsm;

namespace {

constexpr size_t kScratchBytes = DSM_NOALLOC_SCRATCH_BYTES;

// The scratch.  In host code its name is only a stand-in for the device
// variable, never a device address; the address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// The energy kernel's reduction needs one partial sum per block of its fixed
// grid plus the constraint slot: it must fit the array for every lattice.
static_assert(((FE_MAX_BLOCKS * FE_K * sizeof(double) + 255) / 256) * 256 + 256 <= kScratchBytes,
              "the fixed scratch array no longer holds the energy reduction");

// The array's device address in the current device's context.  Resolved on
// every call: a host-side lookup once the library's device image is loaded
// there (the first call on a device loads it), and always the address of the
// context the kernels will run in, also after a device reset.
cudaError_t scratch_address(void **out) {
  *out = nullptr;
  return cudaGetSymbolAddress(out, g_scratch);
}

}  // namespace

extern "C" dsm_status dsm_fe_energy_grad_noalloc(const dsm_params *p, const float *d_c1,
                                                 const float *d_c2, const unsigned char *d_mask,
                                                 int active, double dP, double kcs, double V0,
                                                 double fg, double *d_energy, float *d_grad,
                                                 double *d_terms, void *cuda_stream) {
  TraceRange trace_range("energy and gradient (K4, no-alloc)");
  if (!p || !d_c1 || !d_c2 || !d_grad) return DSM_E_INVAL;
  if (active != 1 && active != 2) return DSM_E_INVAL;
  if (active == 1 && !d_mask) return DSM_E_INVAL;
  if (p->lattice != DSM_D2Q9 && p->lattice != DSM_D3Q19) return DSM_E_INVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->lattice == DSM_D2Q9 && p->nz != 1))
    return DSM_E_INVAL;
  if ((long long)p->nx * p->ny * p->nz >= (1ll << 31)) return DSM_E_INVAL;
  if (kcs < 0.0) return DSM_E_INVAL;
  double k[3];
  dsm_status s = dsm_kappa(p, k);
  if (s != DSM_OK) return s;
  // lattices whose reduction needs more than the fixed array are refused
  if (fe_scratch_bytes(p->lattice, p->nx, p->ny, p->nz) > kScratchBytes) return DSM_E_WORKSPACE;
  FEArgs a;
  s = fe_args_of(p, k, active, fg, &a);
  if (s != DSM_OK) return s;
  void *scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return DSM_E_CUDA;
  a.c1 = d_c1;
  a.c2 = d_c2;
  a.mask = d_mask;
  a.grad = d_grad;
  const cudaError_t e = fe_launch(p->lattice, a, dP, kcs, V0, d_energy, d_terms, scratch,
                                  (cudaStream_t)cuda_stream);
  return e == cudaSuccess ? DSM_OK : DSM_E_CUDA;
}
