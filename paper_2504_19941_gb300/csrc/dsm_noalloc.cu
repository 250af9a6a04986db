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

#include <mutex>

#include "dsm_em.cuh"
#include "dsm_trace.cuh"

using namespace dsm;

namespace {

constexpr size_t kScratchBytes = DSM_NOALLOC_SCRATCH_BYTES;

// The scratch.  In host code its name is only a stand-in for the device
// variable, never a device address; the address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices];  // device address of g_scratch, per device, once resolved

// Set-up, once per device, with that device current: resolve the device
// address of the scratch array.
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" dsm_status dsm_fe_energy_grad_noalloc(const dsm_params *p, const float *d_c1,
                                                 const float *d_c2, const unsigned char *d_mask,
                                                 int active, double dP, double kcs, double V0,
                                                 double fg, double *d_energy, float *d_grad,
                                                 double *d_terms, void *cuda_stream) {
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
  return fe_launch(p->lattice, a, dP, kcs, V0, d_energy, d_terms, scratch,
                   (cudaStream_t)cuda_stream) == cudaSuccess
             ? DSM_OK
             : DSM_E_CUDA;
}
