// dsm_abi.cu -- the extern "C" entry points declared in include/dsm.h.
// Host code only: argument checks, workspace carving, dispatch to the typed
// kernels, error latching.  No device memory is ever allocated here.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "dsm_em.cuh"
#include "dsm_lb_impl.cuh"
#include "dsm_tmap.cuh"
#include "dsm_trace.cuh"

using namespace dsm;

struct dsm_lattice {
  dsm_params prm;
  double kappa[3];
  LBTable tab;
  int kind, q;
  long long N, pitch;
  char *ws;
  size_t ws_bytes;
  void *f[2], *g[2];
  float *g0[2];
  void *Cb[2];   // Cb[cur]: C of the state's last collision; Cb[cur ^ 1]: moments output
  void *M;       // g held as g_eq: A, u_x, u_y, u_z planes
  void *C1;
  unsigned char *mask;
  double *partials, *obs;
  int *err;
  long long obs_blocks;
  int cur;
  cudaStream_t stream;
  long long step;
  bool has_solid, has_fluid, latched, moments_ready;
  int g_form;      // DSM_G_AUTO or DSM_G_POPULATIONS
  bool eq;         // the fused pass stores g as g_eq (tau_g = 1 and DSM_G_AUTO)
  bool g_implicit; // the current g are held as g_eq
  StepParams sp;
  // single-pass step (dsm_zstep.cuh): padded quads (A, C, u_x, u_y) and u_z,
  // two buffers, and padded C1; zc: the buffer holding the current state while
  // zpacked
  bool zok;        // the workspace has the padded buffers (D3Q19, nx % 32, ny % 8, tau_g = 1, periodic)
  bool zpacked;    // the current g_eq state lives in the padded buffers
  bool zmaps_ok;   // maps[] encoded
  int zc, nxp, nyp;
  void *Qz[2], *Uz[2], *C1z;
  ZMaps maps[2];   // maps[b]: read the padded state of buffer b (and C1)
  int step_form;   // DSM_STEP_AUTO or DSM_STEP_TWO_PASS
  int zrun;        // planes per block of the single-pass step (0: automatic)
  int zrun_auto;
  // observables ring (dsm_set_observables_ring): caller-owned device records,
  // one appended by dsm_step after each step that is a multiple of ring_every
  double *ring = nullptr;
  int ring_cap = 0;
  long long ring_every = 0, ring_count = 0;
};

namespace {


dsm_status cuda_status(cudaError_t e) { return e == cudaSuccess ? DSM_OK : DSM_E_CUDA; }

// Polls of a bounded device wait before it gives up (dsm_set_wait_limit);
// 0: each kernel's default.
unsigned long long g_wait_limit = 0;

bool lb_table_for(int kind, int precision, LBTable *t) {
  switch (precision) {
    case DSM_F64: *t = lb_table_f64(kind); return true;
    case DSM_F32: *t = lb_table_f32(kind); return true;
    case DSM_BF16_STORE: *t = lb_table_bf16(kind); return true;
    case DSM_F16_STORE: *t = lb_table_f16(kind); return true;
    default: return false;
  }
}

// Tensions -> kappa (Sec. II.A, Eq. [frozen:kappa]); tension_mode 1 first
// applies Young's relation gamma_13 = gamma_12 + gamma_23 cos(theta).
dsm_status kappa_of(const dsm_params *p, double k[3]) {
  if (!(p->alpha > 0.0)) return DSM_E_INVAL;
  double g12 = p->g12, g23 = p->g23, g13 = p->g13;
  if (p->tension_mode == 1) g13 = g12 + g23 * cos(p->theta_deg * 3.14159265358979323846 / 180.0);
  else if (p->tension_mode != 0) return DSM_E_INVAL;
  k[0] = 3.0 / p->alpha * (g12 + g13 - g23);
  k[1] = 3.0 / p->alpha * (g12 - g13 + g23);
  k[2] = 3.0 / p->alpha * (-g12 + g13 + g23);
  if (!(k[1] > 0.0) || !(k[2] > 0.0)) return DSM_E_INVAL;
  return DSM_OK;
}

dsm_status check_params(const dsm_params *p) {
  if (!p) return DSM_E_INVAL;
  if (p->lattice != DSM_D2Q9 && p->lattice != DSM_D3Q19) return DSM_E_INVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return DSM_E_INVAL;
  if (p->lattice == DSM_D2Q9 && p->nz != 1) return DSM_E_INVAL;
  if ((long long)p->nx * p->ny * p->nz >= (1ll << 31)) return DSM_E_INVAL;
  if (p->precision < DSM_F64 || p->precision > DSM_F16_STORE) return DSM_E_INVAL;
  if (!(p->tau2 > 0.5) || !(p->tau3 > 0.5) || !(p->tau_g > 0.5)) return DSM_E_INVAL;
  if (!(p->rho2 > 0.0) || !(p->rho3 > 0.0)) return DSM_E_INVAL;
  if (p->alpha_s < 0.0) return DSM_E_INVAL;
  if (!faces_valid(p)) return DSM_E_INVAL;
  double k[3];
  return kappa_of(p, k);
}

struct Layout {
  size_t f[2], g[2], g0[2], C[2], M, C1, mask, partials, obs, err, Qz[2], Uz[2], C1z, total;
};

// The single-pass step applies to D3Q19 lattices at least one 32 x 8 tile wide
// (the last tiles may be ragged), with tau_g = 1 (g held as g_eq) and periodic
// faces.
bool z_eligible(const dsm_params *p) {
  if (p->lattice != DSM_D3Q19 || p->tau_g != 1.0 || has_walls(p)) return false;
  return z_tiles(p->nx, p->ny);
}
long long z_padded_nodes(const dsm_params *p) {
  return (long long)z_padded_x(p->nx) * z_padded_y(p->ny) * p->nz;
}

long long obs_blocks_of(int kind, int nx, int ny, int nz) {
  const dim3 g = lb_grid(kind, nx, ny, nz);
  return (long long)g.x * g.y * g.z;
}

Layout layout_of(const dsm_params *p, const LBTable &t, long long N, long long pitch) {
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += (size_t)round_up((long long)bytes, 256);
    return at;
  };
  const size_t pop = (size_t)t.q * pitch * t.store_bytes;
  L.f[0] = take(pop);
  L.f[1] = take(pop);
  L.g[0] = take(pop);
  L.g[1] = take(pop);
  L.g0[0] = take(t.k16 ? pitch * sizeof(float) : 0);
  L.g0[1] = take(t.k16 ? pitch * sizeof(float) : 0);
  L.C[0] = take(pitch * t.real_bytes);
  L.C[1] = take(pitch * t.real_bytes);
  L.M = take(4 * pitch * t.real_bytes);
  L.C1 = take(pitch * t.real_bytes);
  L.mask = take(pitch);
  L.partials = take(obs_blocks_of(p->lattice, p->nx, p->ny, p->nz) * OBS_K * sizeof(double));
  L.obs = take(8 * sizeof(double));
  L.err = take(sizeof(int) * 4);
  const long long P = z_eligible(p) ? z_padded_nodes(p) : 0;
  L.Qz[0] = take(4 * P * t.real_bytes);
  L.Qz[1] = take(4 * P * t.real_bytes);
  L.Uz[0] = take(P * t.real_bytes);
  L.Uz[1] = take(P * t.real_bytes);
  L.C1z = take(P * t.real_bytes);
  L.total = o;
  (void)N;
  return L;
}

StepParams step_params(const dsm_params *p, const double k[3]) {
  StepParams s;
  s.kappa1 = k[0];
  s.kappa2 = k[1];
  s.kappa3 = k[2];
  s.a2 = p->alpha * p->alpha;
  s.alpha_s = p->alpha_s > 0.0 ? p->alpha_s : p->alpha;
  s.rho2 = p->rho2;
  s.rho3 = p->rho3;
  s.tau2 = p->tau2;
  s.tau3 = p->tau3;
  s.tau_g = p->tau_g;
  for (int a = 0; a < 3; a++) s.body[a] = p->body_force[a];
  if (p->lattice == DSM_D2Q9) s.body[2] = 0.0;
  s.beta = p->beta;
  s.omega = p->omega;
  s.rho_contrast = p->rho2 != p->rho3;
  s.walls = 0;
  for (int f = 0; f < 6; f++) {
    s.face[f] = p->face[f];
    s.walls |= p->face[f] != DSM_FACE_PERIODIC;
  }
  return s;
}

LBRaw raw_of(const dsm_lattice *h, int src) {
  LBRaw r;
  memset(&r, 0, sizeof(r));
  r.nx = h->prm.nx;
  r.ny = h->prm.ny;
  r.nz = h->prm.nz;
  r.N = h->N;
  r.pitch = h->pitch;
  r.f_in = h->f[src];
  r.g_in = h->g[src];
  r.g0_in = h->g0[src];
  r.f_out = h->f[src ^ 1];
  r.g_out = h->g[src ^ 1];
  r.g0_out = h->g0[src ^ 1];
  r.C = h->Cb[src ^ 1];
  r.Cprev = h->Cb[src];
  r.M = h->M;
  r.nxp = h->nxp;
  r.nyp = h->nyp;
  r.eq = h->eq;
  r.implicit = h->g_implicit;
  r.C1 = h->C1;
  r.mask = h->mask;
  r.partials = h->partials;
  r.err = h->err;
  r.p = h->sp;
  return r;
}

// ---- single-pass step -------------------------------------------------------
bool z_maps(dsm_lattice *h) {
  if (h->zmaps_ok) return true;
  const int rb = h->tab.real_bytes, nz = h->prm.nz;
  for (int b = 0; b < 2; b++) {
    if (!encode_plane_map(&h->maps[b].Q, h->Qz[b], rb, 4, h->nxp, h->nyp, nz, ZB_Y) ||
        !encode_plane_map(&h->maps[b].U, h->Uz[b], rb, 1, h->nxp, h->nyp, nz, ZB_Y) ||
        !encode_plane_map(&h->maps[b].C1, h->C1z, rb, 1, h->nxp, h->nyp, nz, ZB1_Y))
      return false;
  }
  h->zmaps_ok = true;
  return true;
}

// The longest-lasting choice of planes per block: runs of zr planes give
// tiles * ceil(nz / zr) blocks, which run in waves of the resident blocks; a
// wave lasts about zr planes plus the run's prologue (this step's C of two
// extra planes and the first staged planes, about 0.7 of a plane).
int z_auto_run(dsm_lattice *h) {
  if (h->zrun_auto) return h->zrun_auto;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long resident = (long long)(sms > 0 ? sms : 152) * (h->tab.zresident() > 0 ? h->tab.zresident() : 1);
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

bool z_active(const dsm_lattice *h) {
  return h->zok && h->eq && h->step_form == DSM_STEP_AUTO;
}

// Canonical g_eq state -> padded buffers (buffer 0), and padded C1.
cudaError_t z_pack(dsm_lattice *h) {
  if (!z_maps(h)) return cudaErrorInvalidValue;
  LBRaw a = raw_of(h, h->cur);
  cudaError_t e = h->tab.zpack(a, h->Qz[0], h->Qz[1], h->Uz[0], h->Uz[1], h->C1z, h->stream);
  if (e != cudaSuccess) return e;
  h->zc = 0;
  h->zpacked = true;
  return cudaSuccess;
}

// Padded state -> canonical g_eq state (A, u planes and C of the last
// collision), before any call that reads the state in its canonical layout.
cudaError_t z_unpack(dsm_lattice *h) {
  if (!h->zpacked) return cudaSuccess;
  LBRaw a = raw_of(h, h->cur);
  cudaError_t e = h->tab.zunpack(a, h->Qz[h->zc], h->Uz[h->zc], h->Cb[h->cur], h->stream);
  if (e != cudaSuccess) return e;
  h->zpacked = false;
  return cudaSuccess;
}

// Read and clear nothing: report the latched device error word.
dsm_status read_err(dsm_lattice *h, int *word) {
  int w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return DSM_E_CUDA;
  *word = w;
  return DSM_OK;
}

}  // namespace

// Final deterministic reduction of the observables' block partials.
__global__ void obs_finalize_kernel(const double *partials, long long nb, double *out) {
  __shared__ double sh[OBS_K][256];
  double s[OBS_K] = {0, 0, 0, 0, 0};
  for (long long b = threadIdx.x; b < nb; b += blockDim.x)
    for (int k = 0; k < OBS_K; k++) {
      const double v = partials[b * OBS_K + k];
      s[k] = (k >= 3) ? fmax(s[k], v) : s[k] + v;
    }
  for (int k = 0; k < OBS_K; k++) sh[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int k = 0; k < OBS_K; k++)
        sh[k][threadIdx.x] = (k >= 3) ? fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + st])
                                      : sh[k][threadIdx.x] + sh[k][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < OBS_K) out[threadIdx.x] = sh[threadIdx.x][0];
}

// One observables record (step, then the OBS_K values) into the ring.
__global__ void obs_record_kernel(const double *obs, double *rec, long long step) {
  if (threadIdx.x == 0) rec[0] = (double)step;
  if (threadIdx.x < OBS_K) rec[1 + threadIdx.x] = obs[threadIdx.x];
}

namespace {

// The observables of the current state into h->obs, on the lattice's stream,
// without synchronising: the moments and observables passes over the
// canonical state, then the deterministic final reduction.
cudaError_t obs_launch(dsm_lattice *h) {
  cudaError_t e = z_unpack(h);
  if (e != cudaSuccess) return e;
  LBRaw a = raw_of(h, h->cur);
  e = h->tab.moments(a, h->stream);
  if (e == cudaSuccess) e = h->tab.node(a, 2, MODE_OBS, h->stream);
  if (e != cudaSuccess) return e;
  obs_finalize_kernel<<<1, 256, 0, h->stream>>>(h->partials, h->obs_blocks, h->obs);
  return cudaGetLastError();
}

}  // namespace

// S = {C1 > 1/2} (dsm_solid_region)
template <class T>
__global__ void __launch_bounds__(256) solid_region_kernel(const T *c1, unsigned char *mask,
                                                           long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    mask[k] = c1[k] > T(0.5) ? 1 : 0;
}

extern "C" {

int dsm_checked_build(void) {
#ifdef DSM_CHECKED
  return 1;
#else
  return 0;
#endif
}

const char *dsm_status_string(dsm_status s) {
  switch (s) {
    case DSM_OK: return "ok";
    case DSM_E_INVAL: return "invalid argument";
    case DSM_E_WORKSPACE: return "workspace too small or misaligned";
    case DSM_E_CUDA: return "CUDA error";
    case DSM_E_NONFINITE: return "non-finite population";
    case DSM_E_TIMEOUT: return "device wait timed out";
    case DSM_E_STATE: return "call out of order or handle latched in error";
    case DSM_E_UNSUPPORTED: return "unsupported";
    case DSM_E_BOUNDS: return "index out of bounds (checked build)";
  }
  return "unknown status";
}

dsm_status dsm_lattice_table(int lattice, int *q_out, int *c_out, double *w_out) {
  if (!q_out || !c_out || !w_out) return DSM_E_INVAL;
  if (lattice == DSM_D2Q9) {
    *q_out = 9;
    for (int i = 0; i < 9; i++) {
      c_out[3 * i] = Lat<0>::cx(i);
      c_out[3 * i + 1] = Lat<0>::cy(i);
      c_out[3 * i + 2] = 0;
      w_out[i] = Lat<0>::w(i);
    }
    return DSM_OK;
  }
  if (lattice == DSM_D3Q19) {
    *q_out = 19;
    for (int i = 0; i < 19; i++) {
      c_out[3 * i] = Lat<1>::cx(i);
      c_out[3 * i + 1] = Lat<1>::cy(i);
      c_out[3 * i + 2] = Lat<1>::cz(i);
      w_out[i] = Lat<1>::w(i);
    }
    return DSM_OK;
  }
  return DSM_E_INVAL;
}

dsm_status dsm_kappa(const dsm_params *p, double kappa_out[3]) {
  if (!p || !kappa_out) return DSM_E_INVAL;
  return kappa_of(p, kappa_out);
}

dsm_status dsm_workspace_bytes(const dsm_params *p, size_t *bytes) {
  dsm_status s = check_params(p);
  if (s != DSM_OK) return s;
  if (!bytes) return DSM_E_INVAL;
  LBTable t;
  lb_table_for(p->lattice, p->precision, &t);
  const long long N = (long long)p->nx * p->ny * p->nz;
  *bytes = layout_of(p, t, N, round_up(N, 64)).total;
  return DSM_OK;
}

dsm_status dsm_create(const dsm_params *p, void *d_workspace, size_t bytes, void *cuda_stream,
                      dsm_lattice **out) {
  if (!out) return DSM_E_INVAL;
  *out = nullptr;
  dsm_status s = check_params(p);
  if (s != DSM_OK) return s;
  LBTable t;
  lb_table_for(p->lattice, p->precision, &t);
  const long long N = (long long)p->nx * p->ny * p->nz;
  const long long pitch = round_up(N, 64);
  Layout L = layout_of(p, t, N, pitch);
  if (!d_workspace || bytes < L.total || ((uintptr_t)d_workspace & 255u)) return DSM_E_WORKSPACE;
  dsm_lattice *h = new (std::nothrow) dsm_lattice;
  if (!h) return DSM_E_INVAL;
  memset(h, 0, sizeof(*h));
  h->prm = *p;
  kappa_of(p, h->kappa);
  h->tab = t;
  h->kind = p->lattice;
  h->q = t.q;
  h->N = N;
  h->pitch = pitch;
  h->ws = (char *)d_workspace;
  h->ws_bytes = bytes;
  for (int b = 0; b < 2; b++) {
    h->f[b] = h->ws + L.f[b];
    h->g[b] = h->ws + L.g[b];
    h->g0[b] = t.k16 ? (float *)(h->ws + L.g0[b]) : nullptr;
  }
  h->Cb[0] = h->ws + L.C[0];
  h->Cb[1] = h->ws + L.C[1];
  h->M = h->ws + L.M;
  h->C1 = h->ws + L.C1;
  h->mask = (unsigned char *)(h->ws + L.mask);
  h->partials = (double *)(h->ws + L.partials);
  h->obs = (double *)(h->ws + L.obs);
  h->err = (int *)(h->ws + L.err);
  h->obs_blocks = obs_blocks_of(p->lattice, p->nx, p->ny, p->nz);
  h->zok = z_eligible(p);
  h->nxp = z_padded_x(p->nx);
  h->nyp = z_padded_y(p->ny);
  for (int b = 0; b < 2; b++) {
    h->Qz[b] = h->zok ? h->ws + L.Qz[b] : nullptr;
    h->Uz[b] = h->zok ? h->ws + L.Uz[b] : nullptr;
  }
  h->C1z = h->zok ? h->ws + L.C1z : nullptr;
  h->step_form = DSM_STEP_AUTO;
  h->stream = (cudaStream_t)cuda_stream;
  h->sp = step_params(p, h->kappa);
  h->g_form = DSM_G_AUTO;
  h->eq = p->tau_g == 1.0 && !has_walls(p);
  // no solid yet: C1 = 0 everywhere; clear the error word and the mask
  cudaError_t e = cudaMemsetAsync(h->C1, 0, pitch * t.real_bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->mask, 0, pitch, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int) * 4, h->stream);
  if (e != cudaSuccess) {
    delete h;
    return DSM_E_CUDA;
  }
  *out = h;
  return DSM_OK;
}

dsm_status dsm_set_solid(dsm_lattice *h, const void *d_field, int kind) {
  if (!h || !d_field) return DSM_E_INVAL;
  cudaError_t e;
  if (kind == 0) e = h->tab.solid(d_field, h->C1, h->N, h->sp.alpha_s, h->stream);
  else if (kind == 1)
    e = cudaMemcpyAsync(h->C1, d_field, h->N * h->tab.real_bytes, cudaMemcpyDeviceToDevice, h->stream);
  else return DSM_E_INVAL;
  if (e != cudaSuccess) return DSM_E_CUDA;
  h->has_solid = true;
  h->has_fluid = false;
  h->zpacked = false;
  return DSM_OK;
}

dsm_status dsm_relax_solid(dsm_lattice *h, const unsigned char *d_mask, int steps, double beta,
                           double omega) {
  TraceRange trace_range("dsm_relax_solid (stage 1)");
  if (!h || !d_mask || steps < 0 || beta < 0.0 || omega < 0.0) return DSM_E_INVAL;
  cudaError_t e = cudaMemcpyAsync(h->mask, d_mask, h->N, cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return DSM_E_CUDA;
  h->sp.beta = beta;
  h->sp.omega = omega;
  // initial state of stage 1 from the current C1, written into buffer 0
  // (stage 1 keeps g as populations)
  h->cur = 0;
  h->g_implicit = false;
  h->has_fluid = false;
  h->zpacked = false;
  LBRaw r = raw_of(h, 1);  // out = buffer 0
  r.eq = 0;
  if ((e = h->tab.init(r, h->C1, 1, h->stream)) != cudaSuccess) return DSM_E_CUDA;
  for (int t = 0; t < steps; t++) {
    LBRaw a = raw_of(h, h->cur);
    a.eq = 0;
    if ((e = h->tab.moments(a, h->stream)) != cudaSuccess) return DSM_E_CUDA;
    if ((e = h->tab.node(a, 1, MODE_STEP, h->stream)) != cudaSuccess) return DSM_E_CUDA;
    h->cur ^= 1;
  }
  // relaxed C1 = the concentration the next step would see
  LBRaw a = raw_of(h, h->cur);
  if ((e = h->tab.moments(a, h->stream)) != cudaSuccess) return DSM_E_CUDA;
  e = cudaMemcpyAsync(h->C1, a.C, h->N * h->tab.real_bytes, cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return DSM_E_CUDA;
  h->sp.beta = h->prm.beta;
  h->sp.omega = h->prm.omega;
  h->has_solid = true;
  h->has_fluid = false;
  return DSM_OK;
}

dsm_status dsm_solid_region(dsm_lattice *h, unsigned char *d_mask) {
  if (!h || !d_mask) return DSM_E_INVAL;
  if (!h->has_solid) return DSM_E_STATE;
  long long blocks = (h->N + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (h->tab.real_bytes == 8)
    solid_region_kernel<double><<<(int)blocks, 256, 0, h->stream>>>((const double *)h->C1, d_mask,
                                                                    h->N);
  else
    solid_region_kernel<float><<<(int)blocks, 256, 0, h->stream>>>((const float *)h->C1, d_mask,
                                                                   h->N);
  return cuda_status(cudaGetLastError());
}

dsm_status dsm_set_fluid(dsm_lattice *h, const void *d_c2) {
  if (!h || !d_c2) return DSM_E_INVAL;
  h->cur = 0;
  LBRaw r = raw_of(h, 1);  // writes buffer 0
  cudaError_t e = h->tab.init(r, d_c2, 2, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int) * 4, h->stream);
  if (e != cudaSuccess) return DSM_E_CUDA;
  h->step = 0;
  h->has_fluid = true;
  h->latched = false;
  h->moments_ready = false;
  h->g_implicit = false;  // the initial g are written as populations
  h->zpacked = false;
  return DSM_OK;
}

dsm_status dsm_step(dsm_lattice *h, long long nsteps) {
  TraceRange trace_range("dsm_step");
  if (!h || nsteps < 0) return DSM_E_INVAL;
  if (!h->has_fluid || h->latched) return DSM_E_STATE;
  const bool single = z_active(h);
  if (!single && z_unpack(h) != cudaSuccess) return DSM_E_CUDA;
  for (long long t = 0; t < nsteps; t++) {
    cudaError_t e;
    if (single && h->g_implicit) {
      // one pass per step over the padded g_eq state
      if (!h->zpacked && (e = z_pack(h)) != cudaSuccess) return DSM_E_CUDA;
      LBRaw a = raw_of(h, h->cur);
      a.Qz = h->Qz[h->zc ^ 1];
      a.Uz = h->Uz[h->zc ^ 1];
      e = h->tab.zstep(a, h->maps[h->zc], h->zrun > 0 ? h->zrun : z_auto_run(h), h->stream);
      if (e != cudaSuccess) return DSM_E_CUDA;
      h->zc ^= 1;
    } else {
      // moments pass, then the fused pass (also the first step after
      // dsm_set_fluid, whose g are populations)
      LBRaw a = raw_of(h, h->cur);
      e = h->tab.moments(a, h->stream);
      if (e == cudaSuccess) e = h->tab.node(a, 2, MODE_STEP, h->stream);
      if (e != cudaSuccess) return DSM_E_CUDA;
    }
    h->cur ^= 1;
    h->step++;
    h->g_implicit = h->eq;
    if (h->ring && h->step % h->ring_every == 0) {
      // observables record into the ring: device work only, no synchronisation
      if ((e = obs_launch(h)) != cudaSuccess) return DSM_E_CUDA;
      double *rec = h->ring + (h->ring_count % h->ring_cap) * DSM_OBS_RECORD;
      obs_record_kernel<<<1, 32, 0, h->stream>>>(h->obs, rec, h->step);
      if ((e = cudaGetLastError()) != cudaSuccess) return DSM_E_CUDA;
      h->ring_count++;
    }
  }
  h->moments_ready = false;
  return DSM_OK;
}

dsm_status dsm_set_observables_ring(dsm_lattice *h, double *d_ring, int capacity,
                                    long long every) {
  if (!h) return DSM_E_INVAL;
  if (!d_ring || every == 0) {
    h->ring = nullptr;
    h->ring_cap = 0;
    h->ring_every = 0;
    h->ring_count = 0;
    return DSM_OK;
  }
  if (capacity < 1 || every < 0 || ((uintptr_t)d_ring & 7u)) return DSM_E_INVAL;
  h->ring = d_ring;
  h->ring_cap = capacity;
  h->ring_every = every;
  h->ring_count = 0;
  return DSM_OK;
}

dsm_status dsm_observables_ring_count(const dsm_lattice *h, long long *written) {
  if (!h || !written) return DSM_E_INVAL;
  *written = h->ring_count;
  return DSM_OK;
}

dsm_status dsm_set_body_force(dsm_lattice *h, const double *body) {
  if (!h || !body) return DSM_E_INVAL;
  for (int a = 0; a < 3; a++)
    if (!isfinite(body[a])) return DSM_E_INVAL;
  for (int a = 0; a < 3; a++) h->prm.body_force[a] = body[a];
  h->sp.body[0] = body[0];
  h->sp.body[1] = body[1];
  h->sp.body[2] = h->kind == DSM_D2Q9 ? 0.0 : body[2];
  return DSM_OK;
}

dsm_status dsm_set_step_form(dsm_lattice *h, int form, int zrun) {
  if (!h || (form != DSM_STEP_AUTO && form != DSM_STEP_TWO_PASS) || zrun < 0) return DSM_E_INVAL;
  if (form == DSM_STEP_TWO_PASS && z_unpack(h) != cudaSuccess) return DSM_E_CUDA;
  h->step_form = form;
  h->zrun = zrun;
  return DSM_OK;
}

dsm_status dsm_step_info(dsm_lattice *h, int *single_pass, int *zrun) {
  if (!h) return DSM_E_INVAL;
  const bool single = z_active(h);
  if (single_pass) *single_pass = single ? 1 : 0;
  if (zrun) *zrun = single ? (h->zrun > 0 ? h->zrun : z_auto_run(h)) : 0;
  return DSM_OK;
}

dsm_status dsm_step_moments(dsm_lattice *h) {
  TraceRange trace_range("moments pass (K1)");
  if (!h) return DSM_E_INVAL;
  if (!h->has_fluid || h->latched) return DSM_E_STATE;
  if (z_unpack(h) != cudaSuccess) return DSM_E_CUDA;
  LBRaw a = raw_of(h, h->cur);
  if (h->tab.moments(a, h->stream) != cudaSuccess) return DSM_E_CUDA;
  h->moments_ready = true;
  return DSM_OK;
}

dsm_status dsm_step_collide(dsm_lattice *h) {
  TraceRange trace_range("fused pass (K2)");
  if (!h) return DSM_E_INVAL;
  if (!h->has_fluid || h->latched || !h->moments_ready) return DSM_E_STATE;
  if (z_unpack(h) != cudaSuccess) return DSM_E_CUDA;
  LBRaw a = raw_of(h, h->cur);
  if (h->tab.node(a, 2, MODE_STEP, h->stream) != cudaSuccess) return DSM_E_CUDA;
  h->cur ^= 1;
  h->step++;
  h->g_implicit = h->eq;
  h->moments_ready = false;
  return DSM_OK;
}

dsm_status dsm_get_observables(dsm_lattice *h, dsm_observables *out) {
  if (!h || !out) return DSM_E_INVAL;
  if (!h->has_fluid) return DSM_E_STATE;
  cudaError_t e = obs_launch(h);
  if (e != cudaSuccess) return DSM_E_CUDA;
  double v[OBS_K];
  e = cudaMemcpyAsync(v, h->obs, sizeof(v), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return DSM_E_CUDA;
  int word = 0;
  dsm_status s = read_err(h, &word);  // synchronises
  if (s != DSM_OK) return s;
  out->mass_c2 = v[0];
  out->mass_c1 = v[1];
  out->kinetic = v[2];
  out->max_u = v[3];
  out->step = h->step;
  out->nonfinite = (v[4] > 0.0 || (word & ERR_NONFINITE)) ? 1 : 0;
  if (word & ERR_TIMEOUT) {
    h->latched = true;
    return DSM_E_TIMEOUT;
  }
  if (word & ERR_BOUNDS) {
    h->latched = true;
    return DSM_E_BOUNDS;
  }
  if (out->nonfinite) {
    h->latched = true;
    return DSM_E_NONFINITE;
  }
  return DSM_OK;
}

dsm_status dsm_get_field(dsm_lattice *h, int field, void *d_dst) {
  if (!h || !d_dst || field < DSM_FIELD_C1 || field > DSM_FIELD_TAU) return DSM_E_INVAL;
  cudaError_t e;
  if (field == DSM_FIELD_C1) {
    e = cudaMemcpyAsync(d_dst, h->C1, h->N * h->tab.real_bytes, cudaMemcpyDeviceToDevice, h->stream);
    return cuda_status(e);
  }
  if (!h->has_fluid) return DSM_E_STATE;
  if (z_unpack(h) != cudaSuccess) return DSM_E_CUDA;
  LBRaw a = raw_of(h, h->cur);
  a.out = d_dst;
  a.field_sel = field;
  e = h->tab.moments(a, h->stream);
  if (e == cudaSuccess) e = h->tab.node(a, 2, MODE_FIELDS, h->stream);
  return cuda_status(e);
}

dsm_status dsm_get_populations(dsm_lattice *h, void *d_f, void *d_g) {
  if (!h || !d_f || !d_g) return DSM_E_INVAL;
  if (!h->has_fluid) return DSM_E_STATE;
  if (z_unpack(h) != cudaSuccess) return DSM_E_CUDA;
  LBRaw a = raw_of(h, h->cur);
  return cuda_status(h->tab.get_pops(a, d_f, d_g, h->stream));
}

dsm_status dsm_set_populations(dsm_lattice *h, const void *d_f, const void *d_g) {
  if (!h || !d_f || !d_g) return DSM_E_INVAL;
  LBRaw a = raw_of(h, h->cur ^ 1);  // out = current buffer
  cudaError_t e = h->tab.set_pops(a, d_f, d_g, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int) * 4, h->stream);
  if (e != cudaSuccess) return DSM_E_CUDA;
  h->has_fluid = true;
  h->latched = false;
  h->moments_ready = false;
  h->g_implicit = false;
  h->zpacked = false;
  return DSM_OK;
}

dsm_status dsm_set_g_storage(dsm_lattice *h, int form) {
  if (!h || (form != DSM_G_AUTO && form != DSM_G_POPULATIONS)) return DSM_E_INVAL;
  const bool eq = form == DSM_G_AUTO && h->prm.tau_g == 1.0 && !has_walls(&h->prm);
  if (z_unpack(h) != cudaSuccess) return DSM_E_CUDA;
  if (h->g_implicit && !eq) {
    // write the current g_eq out as populations of the current buffer
    LBRaw a = raw_of(h, h->cur ^ 1);  // g_out = current buffer
    a.Cprev = h->Cb[h->cur];
    if (h->tab.materialize(a, h->stream) != cudaSuccess) return DSM_E_CUDA;
    h->g_implicit = false;
    h->moments_ready = false;
  }
  h->g_form = form;
  h->eq = eq;
  return DSM_OK;
}

dsm_status dsm_get_g_storage(dsm_lattice *h, int *form, int *implicit_now) {
  if (!h) return DSM_E_INVAL;
  if (form) *form = h->g_form;
  if (implicit_now) *implicit_now = h->g_implicit ? 1 : 0;
  return DSM_OK;
}

// Raw state (checkpoint): a 256-byte header, then the current buffer's f, g,
// 16-bit g_0, C of the last collision and the g_eq planes, each region
// 256-byte aligned.  Restoring it continues the run bitwise.
namespace {
constexpr unsigned kStateMagic = 0x53534d44u;  // "DSMS"
struct StateHeader {
  unsigned magic, version;
  int lattice, precision, nx, ny, nz, implicit;
  long long step, pitch;
};
struct StateLayout {
  size_t f, g, g0, C, M, total;
};
StateLayout state_layout(const dsm_lattice *h) {
  StateLayout L;
  size_t o = 256;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += (size_t)round_up((long long)bytes, 256);
    return at;
  };
  const size_t pop = (size_t)h->q * h->pitch * h->tab.store_bytes;
  L.f = take(pop);
  L.g = take(pop);
  L.g0 = take(h->tab.k16 ? h->pitch * sizeof(float) : 0);
  L.C = take(h->pitch * h->tab.real_bytes);
  L.M = take(4 * h->pitch * h->tab.real_bytes);
  L.total = o;
  return L;
}
}  // namespace

dsm_status dsm_state_bytes(dsm_lattice *h, size_t *bytes) {
  if (!h || !bytes) return DSM_E_INVAL;
  *bytes = state_layout(h).total;
  return DSM_OK;
}

dsm_status dsm_get_state(dsm_lattice *h, void *d_dst, size_t bytes) {
  if (!h || !d_dst) return DSM_E_INVAL;
  if (!h->has_fluid) return DSM_E_STATE;
  const StateLayout L = state_layout(h);
  if (bytes < L.total || ((uintptr_t)d_dst & 255u)) return DSM_E_WORKSPACE;
  if (z_unpack(h) != cudaSuccess) return DSM_E_CUDA;
  StateHeader hd;
  memset(&hd, 0, sizeof(hd));
  hd.magic = kStateMagic;
  hd.version = 1;
  hd.lattice = h->kind;
  hd.precision = h->prm.precision;
  hd.nx = h->prm.nx;
  hd.ny = h->prm.ny;
  hd.nz = h->prm.nz;
  hd.implicit = h->g_implicit ? 1 : 0;
  hd.step = h->step;
  hd.pitch = h->pitch;
  char *d = (char *)d_dst;
  const size_t pop = (size_t)h->q * h->pitch * h->tab.store_bytes;
  const size_t real = h->pitch * h->tab.real_bytes;
  cudaStream_t st = h->stream;
  cudaError_t e = cudaMemcpyAsync(d, &hd, sizeof(hd), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + L.f, h->f[h->cur], pop, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + L.g, h->g[h->cur], pop, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && h->tab.k16)
    e = cudaMemcpyAsync(d + L.g0, h->g0[h->cur], h->pitch * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + L.C, h->Cb[h->cur], real, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + L.M, h->M, 4 * real, cudaMemcpyDeviceToDevice, st);
  // the header copy reads host stack memory
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_status(e);
}

dsm_status dsm_set_state(dsm_lattice *h, const void *d_src, size_t bytes) {
  if (!h || !d_src) return DSM_E_INVAL;
  const StateLayout L = state_layout(h);
  if (bytes < L.total || ((uintptr_t)d_src & 255u)) return DSM_E_WORKSPACE;
  StateHeader hd;
  cudaStream_t st = h->stream;
  cudaError_t e = cudaMemcpyAsync(&hd, d_src, sizeof(hd), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return DSM_E_CUDA;
  if (hd.magic != kStateMagic || hd.version != 1 || hd.lattice != h->kind ||
      hd.precision != h->prm.precision || hd.nx != h->prm.nx || hd.ny != h->prm.ny ||
      hd.nz != h->prm.nz || hd.pitch != h->pitch || (hd.implicit != 0 && hd.implicit != 1) ||
      hd.step < 0)
    return DSM_E_INVAL;
  const char *d = (const char *)d_src;
  const size_t pop = (size_t)h->q * h->pitch * h->tab.store_bytes;
  const size_t real = h->pitch * h->tab.real_bytes;
  e = cudaMemcpyAsync(h->f[0], d + L.f, pop, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->g[0], d + L.g, pop, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && h->tab.k16)
    e = cudaMemcpyAsync(h->g0[0], d + L.g0, h->pitch * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->Cb[0], d + L.C, real, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->M, d + L.M, 4 * real, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int) * 4, st);
  if (e != cudaSuccess) return DSM_E_CUDA;
  h->cur = 0;
  h->step = hd.step;
  h->g_implicit = hd.implicit != 0;
  h->zpacked = false;
  h->has_fluid = true;
  h->latched = false;
  h->moments_ready = false;
  // a state holding g as g_eq, restored into a handle that keeps populations
  if (h->g_implicit && !h->eq) return dsm_set_g_storage(h, h->g_form);
  return DSM_OK;
}

dsm_status dsm_fe_scratch_bytes(int lattice, int nx, int ny, int nz, size_t *bytes) {
  if (!bytes || (lattice != DSM_D2Q9 && lattice != DSM_D3Q19) || nx < 1 || ny < 1 || nz < 1)
    return DSM_E_INVAL;
  if (lattice == DSM_D2Q9 && nz != 1) return DSM_E_INVAL;
  *bytes = fe_scratch_bytes(lattice, nx, ny, nz);
  return DSM_OK;
}

dsm_status dsm_fe_energy_grad(const dsm_params *p, const float *d_c1, const float *d_c2,
                              const unsigned char *d_mask, int active, double dP, double kcs,
                              double V0, double fg, double *d_energy, float *d_grad,
                              double *d_terms, void *d_scratch, size_t scratch_bytes,
                              void *cuda_stream) {
  TraceRange trace_range("energy and gradient (K4)");
  if (!p || !d_c1 || !d_c2 || !d_grad || !d_scratch) return DSM_E_INVAL;
  if (active != 1 && active != 2) return DSM_E_INVAL;
  if (active == 1 && !d_mask) return DSM_E_INVAL;
  if (p->lattice != DSM_D2Q9 && p->lattice != DSM_D3Q19) return DSM_E_INVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->lattice == DSM_D2Q9 && p->nz != 1))
    return DSM_E_INVAL;
  if ((long long)p->nx * p->ny * p->nz >= (1ll << 31)) return DSM_E_INVAL;
  if (kcs < 0.0) return DSM_E_INVAL;
  double k[3];
  dsm_status s = kappa_of(p, k);
  if (s != DSM_OK) return s;
  if (scratch_bytes < fe_scratch_bytes(p->lattice, p->nx, p->ny, p->nz) ||
      ((uintptr_t)d_scratch & 255u))
    return DSM_E_WORKSPACE;
  FEArgs a;
  s = fe_args_of(p, k, active, fg, &a);
  if (s != DSM_OK) return s;
  a.c1 = d_c1;
  a.c2 = d_c2;
  a.mask = d_mask;
  a.grad = d_grad;
  return cuda_status(fe_launch(p->lattice, a, dP, kcs, V0, d_energy, d_terms, d_scratch,
                               (cudaStream_t)cuda_stream));
}

dsm_status dsm_fe_multi_scratch_bytes(int lattice, int nx, int ny, int nz, int nfluid,
                                      size_t *bytes) {
  if (!bytes || (lattice != DSM_D2Q9 && lattice != DSM_D3Q19) || nx < 1 || ny < 1 || nz < 1)
    return DSM_E_INVAL;
  if (nfluid < 2 || nfluid > FEM_MAX_NF + 1) return DSM_E_INVAL;
  *bytes = fe_multi_scratch_bytes(lattice, nx, ny, nz, nfluid - 1);
  return DSM_OK;
}

dsm_status dsm_fe_energy_grad_multi(const dsm_params *p, int nfluid, const double *kappa,
                                    const float *d_c1, const float *d_c, const double *dP,
                                    const double *kcs, const double *V0, double *d_energy,
                                    float *d_grad, double *d_terms, void *d_scratch,
                                    size_t scratch_bytes, void *cuda_stream) {
  TraceRange trace_range("N-fluid energy and gradient");
  if (!d_c1 || !d_c || !d_grad || !d_scratch) return DSM_E_INVAL;
  FEMArgs a;
  FEMCons cons;
  dsm_status s = fem_args_of(p, nfluid, kappa, dP, kcs, V0, &a, &cons);
  if (s != DSM_OK) return s;
  if (scratch_bytes < fe_multi_scratch_bytes(p->lattice, p->nx, p->ny, p->nz, a.nf) ||
      ((uintptr_t)d_scratch & 255u))
    return DSM_E_WORKSPACE;
  a.c1 = d_c1;
  a.c = d_c;
  a.grad = d_grad;
  return cuda_status(fe_multi_launch(p->lattice, a, cons, d_energy, d_terms, d_scratch,
                                     (cudaStream_t)cuda_stream));
}

dsm_status dsm_vec_scratch_bytes(long long n, size_t *bytes) {
  if (!bytes || n < 0) return DSM_E_INVAL;
  *bytes = vec_scratch_bytes(n);
  return DSM_OK;
}

dsm_status dsm_vec_dot(long long n, const float *d_x, const float *d_y, double *d_out,
                       void *d_scratch, size_t scratch_bytes, void *cuda_stream) {
  if (n < 0 || !d_x || !d_y || !d_out || !d_scratch) return DSM_E_INVAL;
  if (scratch_bytes < vec_scratch_bytes(n)) return DSM_E_WORKSPACE;
  return cuda_status(vec_dot(n, d_x, d_y, d_out, nullptr, d_scratch, (cudaStream_t)cuda_stream));
}

dsm_status dsm_vec_axpy_dev(long long n, double sign, const double *d_a, const double *d_b,
                            const float *d_x, float *d_y, void *cuda_stream) {
  if (n < 0 || !d_a || !d_x || !d_y) return DSM_E_INVAL;
  return cuda_status(vec_axpy_dev(n, sign, d_a, d_b, d_x, d_y, (cudaStream_t)cuda_stream));
}

dsm_status dsm_vec_axpby(long long n, double a, const float *d_x, double b, float *d_y,
                         void *cuda_stream) {
  if (n < 0 || !d_x || !d_y) return DSM_E_INVAL;
  return cuda_status(vec_axpby(n, a, d_x, b, d_y, (cudaStream_t)cuda_stream));
}

dsm_status dsm_lbfgs_direction(long long n, int m, const int *order, const float *d_S,
                               const float *d_Y, const double *d_rho, const double *d_gamma,
                               const float *d_g, float *d_r, double *d_alpha, void *d_scratch,
                               size_t scratch_bytes, void *cuda_stream) {
  if (n < 0 || m < 0 || (m > 0 && (!order || !d_S || !d_Y || !d_rho || !d_alpha)) || !d_gamma ||
      !d_g || !d_r || !d_scratch)
    return DSM_E_INVAL;
  if (scratch_bytes < vec_scratch_bytes(n)) return DSM_E_WORKSPACE;
  return cuda_status(lbfgs_direction(n, m, order, d_S, d_Y, d_rho, d_gamma, d_g, d_r, d_alpha,
                                     d_scratch, (cudaStream_t)cuda_stream));
}

dsm_status dsm_vec_dots_scratch_bytes(long long n, int nv, size_t *bytes) {
  if (!bytes || n < 0 || nv < 0) return DSM_E_INVAL;
  *bytes = vec_dots_scratch_bytes(n, nv);
  return DSM_OK;
}

dsm_status dsm_vec_dots(long long n, int nv, const float *d_V, long long stride,
                        const float *d_x, double *d_out, void *d_scratch, size_t scratch_bytes,
                        void *cuda_stream) {
  if (n < 0 || nv < 0 || stride < 0 || (nv > 0 && (!d_V || !d_x || !d_out || !d_scratch)))
    return DSM_E_INVAL;
  if (nv > 1 && stride < n) return DSM_E_INVAL;
  if (scratch_bytes < vec_dots_scratch_bytes(n, nv)) return DSM_E_WORKSPACE;
  return cuda_status(vec_dots(n, nv, d_V, stride, d_x, d_out, d_scratch, (cudaStream_t)cuda_stream));
}

dsm_status dsm_vec_lincomb(long long n, int nv, const float *d_V, long long stride,
                           const double *coef, const float *d_x, double cx, float *d_y,
                           void *cuda_stream) {
  if (n < 0 || nv < 0 || nv > LINCOMB_MAX || stride < 0 || !d_x || !d_y ||
      (nv > 0 && (!d_V || !coef)))
    return DSM_E_INVAL;
  if (nv > 1 && stride < n) return DSM_E_INVAL;
  return cuda_status(vec_lincomb(n, nv, d_V, stride, coef, d_x, cx, d_y, (cudaStream_t)cuda_stream));
}

// Batch admission: common kind, precision, stream and density-contrast flag.
static dsm_status batch_items(dsm_lattice *const *hs, int n, const long long *nsteps,
                              std::vector<BatchRaw> &items) {
  if (!hs || n < 1) return DSM_E_INVAL;
  const dsm_lattice *h0 = hs[0];
  if (!h0) return DSM_E_INVAL;
  items.resize(n);
  for (int i = 0; i < n; i++) {
    const dsm_lattice *h = hs[i];
    if (!h) return DSM_E_INVAL;
    if (has_walls(&h->prm)) return DSM_E_UNSUPPORTED;  // the batched step is periodic
    if (h->kind != h0->kind || h->prm.precision != h0->prm.precision ||
        h->stream != h0->stream || h->sp.rho_contrast != h0->sp.rho_contrast || h->eq != h0->eq)
      return DSM_E_INVAL;
    if (nsteps && (nsteps[i] < 0 || nsteps[i] > (1ll << 30))) return DSM_E_INVAL;
    items[i].r[0] = raw_of(h, 0);
    items[i].r[1] = raw_of(h, 1);
    items[i].nsteps = nsteps ? nsteps[i] : 0;
    items[i].cur0 = h->cur;
  }
  return DSM_OK;
}

dsm_status dsm_batch_scratch_bytes(dsm_lattice *const *hs, int n, size_t *bytes) {
  if (!bytes) return DSM_E_INVAL;
  std::vector<BatchRaw> items;
  dsm_status s = batch_items(hs, n, nullptr, items);
  if (s != DSM_OK) return s;
  *bytes = hs[0]->tab.batch_bytes(items.data(), n);
  return DSM_OK;
}

dsm_status dsm_batch_step(dsm_lattice *const *hs, int n, const long long *nsteps, void *d_scratch,
                          size_t scratch_bytes) {
  TraceRange trace_range("batched step (K9)");
  if (!nsteps || !d_scratch) return DSM_E_INVAL;
  std::vector<BatchRaw> items;
  dsm_status s = batch_items(hs, n, nsteps, items);
  if (s != DSM_OK) return s;
  for (int i = 0; i < n; i++)
    if (!hs[i]->has_fluid || hs[i]->latched) return DSM_E_STATE;
  for (int i = 0; i < n; i++)
    if (z_unpack(hs[i]) != cudaSuccess) return DSM_E_CUDA;
  if (scratch_bytes < hs[0]->tab.batch_bytes(items.data(), n) || ((uintptr_t)d_scratch & 255u))
    return DSM_E_WORKSPACE;
  cudaError_t e = hs[0]->tab.batch(items.data(), n, d_scratch, scratch_bytes,
                                   hs[0]->sp.rho_contrast != 0, hs[0]->eq, g_wait_limit,
                                   hs[0]->stream);
  if (e != cudaSuccess) return DSM_E_CUDA;
  for (int i = 0; i < n; i++) {
    hs[i]->cur ^= (int)(nsteps[i] & 1);
    hs[i]->step += nsteps[i];
    hs[i]->moments_ready = false;
    if (nsteps[i] > 0) hs[i]->g_implicit = hs[i]->eq;
  }
  return DSM_OK;
}

dsm_status dsm_set_wait_limit(unsigned long long polls) {
  g_wait_limit = polls;
  return DSM_OK;
}

dsm_status dsm_destroy(dsm_lattice *h) {
  if (!h) return DSM_E_INVAL;
  delete h;
  return DSM_OK;
}

}  // extern "C"
