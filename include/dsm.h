/*
 * dsm.h -- C ABI of the GB300 Diffuse Solid Method library (libdsm.so).
 *
 * The library implements, on one NVIDIA GB300 (sm_103a), the lattice
 * Boltzmann time step and the free-energy/gradient kernel of the Diffuse Solid
 * Method (Oktasendra, Rennick, Avis, Panter, Kusumaatmaja, "The Diffuse Solid
 * Method for Wetting and Multiphase Fluid Simulations in Complex Geometries"):
 * N = 2 fluids (liquid C2, gas C3) plus a solid component C1 held to a
 * prescribed geometry.
 *
 * Conventions (all entry points)
 *   - Node index n = x + nx*(y + ny*z); nz = 1 for D2Q9.  Each face of the
 *     lattice is periodic, a mirror or a wall (dsm_params.face).
 *   - "real" is double for DSM_F64 lattices and float for every other precision.
 *   - Device pointers (d_*) must point to memory of the current CUDA device and
 *     stay valid for the call (and, for the workspace, until dsm_destroy).
 *     The library NEVER allocates or frees device memory: the caller owns every
 *     buffer (workspace, inputs, outputs).  Host pointers are borrowed for the
 *     duration of the call only.
 *   - Work is enqueued on the caller's stream (a cudaStream_t passed as void*;
 *     NULL = legacy default stream).  Calls that return host values
 *     (dsm_get_observables) synchronise that stream.
 *   - Errors are returned as dsm_status; nothing throws across the ABI.
 *     Device-detected errors (non-finite populations, a persistent-kernel
 *     barrier that timed out) are latched in the workspace and reported by the
 *     next synchronising call; the handle then stays in DSM_E_STATE until
 *     dsm_set_populations, dsm_set_state or dsm_set_fluid resets it.
 *   - One handle belongs to one stream; calls on different handles are
 *     independent.  The library is not thread-safe for one handle.
 */
#ifndef DSM_H
#define DSM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DSM_OK = 0,
  DSM_E_INVAL = 1,       /* bad argument (sizes, parameters, null pointer) */
  DSM_E_WORKSPACE = 2,   /* workspace too small or misaligned */
  DSM_E_CUDA = 3,        /* a CUDA runtime call or launch failed */
  DSM_E_NONFINITE = 4,   /* a NaN/Inf appeared in the populations */
  DSM_E_TIMEOUT = 5,     /* a bounded device wait ran out */
  DSM_E_STATE = 6,       /* call out of order, or handle latched in error */
  DSM_E_UNSUPPORTED = 7, /* a valid request the library does not implement */
  DSM_E_BOUNDS = 8       /* (checked build) a kernel index left its buffer */
} dsm_status;

typedef enum { DSM_D2Q9 = 0, DSM_D3Q19 = 1 } dsm_lattice_kind;

typedef enum {
  DSM_F64 = 0,        /* FP64 populations and arithmetic */
  DSM_F32 = 1,        /* FP32 populations and arithmetic */
  DSM_BF16_STORE = 2, /* BF16 storage of f_i - w_i and g_i (i != 0), FP32 g_0, FP32 math */
  DSM_F16_STORE = 3   /* FP16 storage, otherwise as DSM_BF16_STORE */
} dsm_precision;

/* Problem statement (Sec. II of the paper).  Tensions follow Sec. II.A,
 * Eq. [frozen:kappa]: kappa_1..3 from gamma_12, gamma_13, gamma_23 and the
 * interface width alpha.  tension_mode = 1 gives the contact angle instead:
 * gamma_13 = gamma_12 + gamma_23 cos(theta) (Young, Supp. B Eq. [eq:CA]), so
 * cos(theta) = (kappa_3 - kappa_2)/(kappa_2 + kappa_3) (Eq. [eqn:st_ca]).
 * kappa_2 <= 0 or kappa_3 <= 0 is rejected with DSM_E_INVAL. */
typedef struct dsm_params {
  int lattice;             /* dsm_lattice_kind */
  int nx, ny, nz;          /* lattice size; nz must be 1 for D2Q9; each >= 1 */
  int precision;           /* dsm_precision */
  double alpha;            /* fluid interface width (the paper uses 1) */
  double alpha_s;          /* tanh width given to an analytic solid; 0 => alpha */
  int tension_mode;        /* 0: (g12, g13, g23)  1: (theta_deg, g23, g12) */
  double g12, g13, g23, theta_deg;
  double rho2, rho3;       /* liquid / gas density, Sec. II.B density map */
  double tau2, tau3;       /* liquid / gas BGK relaxation time */
  double tau_g;            /* Cahn-Hilliard relaxation time; M = (tau_g - 1/2)/3 */
  double body_force[3];    /* body force per unit liquid concentration */
  double beta, omega;      /* solid confinement and range penalty, LB stage 1 */
  int face[6];             /* dsm_face of the faces x-, x+, y-, y+, z-, z+ */
} dsm_params;

/* Domain faces (the symmetry and halfway bounce-back boundaries the paper uses
 * besides periodic ones, Sec. III).  A mirror or wall plane lies half a node
 * beyond the edge node.  Both faces of an axis are periodic, or neither; the
 * z faces of a D2Q9 lattice are periodic.  Other values: DSM_E_INVAL.
 *   Stencils (G, L, the energy's pair sums): beyond a mirror or wall face they
 *   see the edge node itself (zero normal gradient; a wall is neutral, the
 *   method wets through the diffuse solid).
 *   Streaming: a population crossing a mirror is reflected specularly (read at
 *   the image node with the normal components of its velocity reversed); one
 *   crossing a wall is bounced back at the node (f and g alike: no slip, no
 *   flux).  A link crossing a wall takes the wall rule whatever lies beyond;
 *   across a mirror the image node counts as the upstream node, so a solid
 *   image takes the interpolated bounce-back.
 *   Lattices with a mirror or wall face keep g as populations (the g_eq form
 *   of dsm_set_g_storage is periodic only) and are refused by dsm_batch_step
 *   with DSM_E_UNSUPPORTED. */
typedef enum { DSM_FACE_PERIODIC = 0, DSM_FACE_MIRROR = 1, DSM_FACE_WALL = 2 } dsm_face;

typedef struct dsm_observables {
  double mass_c2;   /* sum over nodes of C2 (current time level) */
  double mass_c1;   /* sum over nodes of C1 */
  double kinetic;   /* sum over fluid nodes of rho |u|^2 / 2 */
  double max_u;     /* max over nodes of |u| */
  long long step;   /* steps taken since dsm_set_fluid */
  int nonfinite;    /* 1 if a population is NaN or Inf */
} dsm_observables;

typedef struct dsm_lattice dsm_lattice; /* opaque handle (host memory) */

/* Field selectors of dsm_get_field: macroscopic fields at the current time
 * level (the streaming and moment stages of the next step, without collision). */
enum {
  DSM_FIELD_C1 = 0, DSM_FIELD_C2 = 1, DSM_FIELD_C3 = 2, DSM_FIELD_MU = 3,
  DSM_FIELD_UX = 4, DSM_FIELD_UY = 5, DSM_FIELD_UZ = 6,
  DSM_FIELD_PT = 7,   /* pt = P / c_s^2 */
  DSM_FIELD_RHO = 8, DSM_FIELD_TAU = 9
};

/* Status text (static storage; never NULL). */
const char *dsm_status_string(dsm_status s);

/* 1 in the checked build (libdsm_checked.so, compiled with -DDSM_CHECKED), 0
 * in the normal one.  In the checked build every neighbour, pull, store and
 * padded-plane index that the lattice Boltzmann kernels form is tested against
 * its buffer; one outside it latches DSM_E_BOUNDS in the lattice's error word
 * and the access goes to element 0 instead, so the kernel never touches
 * memory outside the buffer.  dsm_get_observables and dsm_ml_check then
 * return DSM_E_BOUNDS, and the handle stays latched as for DSM_E_TIMEOUT.  The
 * checked build runs the same arithmetic; it is slower and exists to test. */
int dsm_checked_build(void);

/* Velocity set and weights of a lattice as this library orders them:
 * c_out[3*i + a], w_out[i] for i < *q (q_out receives 9 or 19).  D2Q9 follows
 * the table printed in Sec. II.B; D3Q19 is the textbook set (the paper gives
 * only D2Q9). */
dsm_status dsm_lattice_table(int lattice, int *q_out, int *c_out, double *w_out);

/* kappa_1, kappa_2, kappa_3 of a parameter set (Sec. II.A Eq. [frozen:kappa]). */
dsm_status dsm_kappa(const dsm_params *p, double kappa_out[3]);

/* Workspace bytes a lattice of these parameters needs (populations, two
 * buffers each; C1; C, two buffers; the four g_eq planes; solid mask;
 * reduction scratch; for lattices the one-pass step applies to (see
 * dsm_set_step_form), padded (A, u, C), two buffers, and padded C1:
 * 11 reals per padded node, (nx + 8, rounded up to a multiple of 4)(ny + 4) nz
 * nodes). */
dsm_status dsm_workspace_bytes(const dsm_params *p, size_t *bytes);

/* Create a handle over a caller-owned device workspace (>= the size above,
 * 256-byte aligned).  No device allocation happens here or later.
 * Returns DSM_E_INVAL for bad sizes or parameters, DSM_E_WORKSPACE for a short
 * or misaligned workspace. */
dsm_status dsm_create(const dsm_params *p, void *d_workspace, size_t bytes,
                      void *cuda_stream, dsm_lattice **out);

/* Set the solid.  kind 0: d_field is a signed distance to the solid region S
 * (positive inside), turned into C1 = 1/2 + tanh(d / (2 alpha_s))/2, the planar
 * profile of Sec. II.A Eq. [frozen:interface_profile].  kind 1: d_field is C1.
 * d_field holds nx*ny*nz reals. */
dsm_status dsm_set_solid(dsm_lattice *h, const void *d_field, int kind);

/* LB stage 1 (Sec. II.B, Eq. [Free Energy1]): relax C1 for `steps` steps with
 * the confining potential of strength beta on the solid region d_mask (bytes,
 * 1 inside S) and the range penalty omega; rho = 1, tau = tau_g = 1.  Starts
 * from the C1 last set, writes the relaxed C1 back.  Uses the population
 * buffers, so call it before dsm_set_fluid. */
dsm_status dsm_relax_solid(dsm_lattice *h, const unsigned char *d_mask, int steps,
                           double beta, double omega);

/* The solid region of the current diffuse solid: d_mask[n] = 1 where
 * C1 > 1/2, else 0 (nx*ny*nz bytes, device, caller-owned).  This is the
 * redefinition step of the two-step solid initialisation for sharp corners
 * (Sec. II.B, after Eq. [frozen:poly-quadratic_lbm]): a short dsm_relax_solid
 * with larger beta and Omega, then S := {C1 > 1/2} by this call, then a
 * further dsm_relax_solid with the new S.  DSM_E_STATE before any solid was
 * set. */
dsm_status dsm_solid_region(dsm_lattice *h, unsigned char *d_mask);

/* Set the liquid field C2 (nx*ny*nz reals) and initialise the populations at
 * rest: f_i = w_i, g_i = g_eq_i(C2, mu(C2), u = 0).  Resets the step counter
 * and any latched error. */
dsm_status dsm_set_fluid(dsm_lattice *h, const void *d_c2);

/* Advance nsteps LB steps (stage 2, Sec. II.B) asynchronously on the stream.
 * Each step: moments pass (C = sum_i g_i after streaming) then the fused pass
 * (mu, forces, pull-streaming with interpolated bounce-back, BGK collision of
 * f and g). */
dsm_status dsm_step(dsm_lattice *h, long long nsteps);

/* The two passes of dsm_step, for callers that interleave their own work or
 * time the passes: dsm_step_moments computes C of the current state (the
 * moments pass); dsm_step_collide then runs the fused pass and advances the
 * state by one step.  dsm_step(h, 1) equals the two calls in this order;
 * dsm_step_collide without a preceding dsm_step_moments on the same state is
 * DSM_E_STATE. */
dsm_status dsm_step_moments(dsm_lattice *h);
dsm_status dsm_step_collide(dsm_lattice *h);

/* Change the body force on the liquid of a live lattice (body[3], per unit
 * liquid concentration, F_g = C2 b: the gravity-like force of Sec. IV that
 * drives the droplet on the sinusoidal surface, and the pressure of a
 * critical-pressure ramp) for the steps enqueued after this call; the state
 * is kept.  D2Q9 ignores body[2].  DSM_E_INVAL for a non-finite component. */
dsm_status dsm_set_body_force(dsm_lattice *h, const double *body);

/* How dsm_step advances a lattice.  The step of Sec. II.B needs C = sum_i g_i
 * of the streamed populations on each node's neighbourhood before it can form
 * mu, so dsm_step normally runs it as the two passes above.  For D3Q19 lattices
 * with nx >= 32, ny >= 8, tau_g = 1 (g held as g_eq, see
 * dsm_set_g_storage) and periodic faces, DSM_STEP_AUTO instead runs each step
 * as ONE pass: blocks march 32 x 8 tiles (the last ones ragged) up runs of z
 * planes, rebuild the C of
 * the step on chip from the staged (A, u, C) of the previous collision and
 * collide.  The results are the same step (the same per-node arithmetic, so
 * equal to the two-pass step up to nothing but FP32 contraction order); the
 * state then lives in padded buffers of the workspace and is converted back
 * before any call that reads it (fields, observables, populations, checkpoint,
 * dsm_batch_step).  DSM_STEP_TWO_PASS always uses the two passes.
 *   zrun: z planes per block of the one-pass step, 0 = chosen from the lattice
 *   size and the GPU's resident blocks (a tuning knob; results do not depend on
 *   it).  DSM_E_INVAL for an unknown form or zrun < 0. */
enum { DSM_STEP_AUTO = 0, DSM_STEP_TWO_PASS = 1 };
dsm_status dsm_set_step_form(dsm_lattice *h, int form, int zrun);

/* Whether dsm_step currently runs the one-pass step (*single_pass = 1) and
 * with how many z planes per block (*zrun; 0 for the two-pass step).  Either
 * pointer may be NULL. */
dsm_status dsm_step_info(dsm_lattice *h, int *single_pass, int *zrun);

/* Observables of the current state; synchronises the stream.  Returns
 * DSM_E_NONFINITE (and sets out->nonfinite) when the state holds a NaN/Inf,
 * DSM_E_TIMEOUT after a timed-out device wait, DSM_E_BOUNDS after an index
 * fault caught by the checked build (dsm_checked_build). */
dsm_status dsm_get_observables(dsm_lattice *h, dsm_observables *out);

/* Observables ring: a time series of the observables kept on the device, so
 * that a long run can be watched without a host synchronisation per sample.
 * d_ring (device, caller-owned, 8-byte aligned, capacity * DSM_OBS_RECORD
 * doubles) receives one record after every step of dsm_step whose step count
 * (dsm_observables.step) is a multiple of `every`.  A record is
 *   { step, mass_c2, mass_c1, kinetic, max_u, nonfinite nodes }
 * as dsm_get_observables computes them (the same kernels, bitwise the same
 * values), written by kernels on the lattice's stream; record k (counted
 * from this call) sits in slot k % capacity, so the ring keeps the last
 * `capacity` records.  dsm_observables_ring_count gives the number of records
 * written so far (host bookkeeping, no synchronisation); read the ring after
 * synchronising the lattice's stream.  Recording does not change the
 * trajectory.  A record does not latch errors: dsm_get_observables reports
 * them.  d_ring NULL or every 0 turns recording off.  Only dsm_step
 * records: the split step (dsm_step_moments / dsm_step_collide) and
 * dsm_batch_step do not.  DSM_E_INVAL: capacity < 1, every < 0, d_ring
 * misaligned. */
#define DSM_OBS_RECORD 6
dsm_status dsm_set_observables_ring(dsm_lattice *h, double *d_ring, int capacity,
                                    long long every);
dsm_status dsm_observables_ring_count(const dsm_lattice *h, long long *written);

/* One macroscopic field (DSM_FIELD_*) into d_dst (nx*ny*nz reals). */
dsm_status dsm_get_field(dsm_lattice *h, int field, void *d_dst);

/* Post-collision populations of the current state as reals, q-major
 * (d_f[i*N + n], d_g[i*N + n], N = nx*ny*nz, q-order of dsm_lattice_table).
 * A state holding g as g_eq (dsm_set_g_storage) returns g_eq_i evaluated from
 * the stored A, u and C in the lattice's arithmetic. */
dsm_status dsm_get_populations(dsm_lattice *h, void *d_f, void *d_g);

/* Replace the state by the given post-collision populations (reals, layout as
 * above); 16-bit precisions encode them.  Clears a latched error.  The state
 * holds g as populations until the next step. */
dsm_status dsm_set_populations(dsm_lattice *h, const void *d_f, const void *d_g);

/* Storage form of the order-parameter populations g (stage 2).
 *
 * The g collision of Sec. II.B relaxes g_i toward g_eq_i with rate 1/tau_g; at
 * tau_g = 1 (the paper's value) it replaces g_i by g_eq_i outright, and g_eq_i
 * is fixed by the node's C, mu and u:
 *   g_eq_i = w_i (mu + C s_i)  (i != 0),  g_eq_0 = C - (1 - w_0) mu + w_0 C s_0.
 * DSM_G_AUTO (the default) then keeps four reals per node (A = mu - 3/2 C u.u,
 * u) instead of the Q populations, and the moments pass rebuilds
 * C = sum_i g_eq_i(x - c_i) from the neighbours' values: the same step up to
 * rounding, with less than half the memory traffic.  With tau_g != 1 AUTO
 * keeps populations.  DSM_G_POPULATIONS always keeps populations.
 *
 * dsm_set_g_storage may be called at any time; switching a state that holds g
 * as g_eq to populations writes them out (on the stream).  dsm_get_g_storage
 * reports the form set and whether the current state holds g as g_eq
 * (either output pointer may be NULL).  DSM_E_INVAL for an unknown form. */
enum { DSM_G_AUTO = 0, DSM_G_POPULATIONS = 1 };
dsm_status dsm_set_g_storage(dsm_lattice *h, int form);
dsm_status dsm_get_g_storage(dsm_lattice *h, int *form, int *implicit_now);

/* Checkpoint of the current state (not in the paper: restart support).
 * dsm_state_bytes gives the size; dsm_get_state copies the state into the
 * caller's device buffer d_dst (256-byte aligned, >= that size): a header
 * (lattice, precision, sizes, step, storage form) and the raw population /
 * g_eq buffers.  dsm_set_state restores such a buffer into a handle of the
 * same lattice, precision and size, clears a latched error, and the run then
 * continues bitwise as the saved one would have.  Both synchronise the stream
 * (the header passes through host memory).  DSM_E_WORKSPACE for a short or
 * misaligned buffer, DSM_E_INVAL for a header that does not match the handle,
 * DSM_E_STATE for dsm_get_state before dsm_set_fluid. */
dsm_status dsm_state_bytes(dsm_lattice *h, size_t *bytes);
dsm_status dsm_get_state(dsm_lattice *h, void *d_dst, size_t bytes);
dsm_status dsm_set_state(dsm_lattice *h, const void *d_src, size_t bytes);

/* Free-energy twin (Sec. II.A, Eqs. [frozen:total_energy], [frozen:bulk_energy],
 * [frozen:interface_energy], [frozen:pressure_const] / [frozen:volume_const],
 * [frozen:poly-quadratic]; Sec. III.B Eq. [frozen:gravitational energy]).
 * Stateless.  FP32 fields, FP64 energy.
 *   E = sum_x [ sum_n kappa_n/2 C_n^2 (1 - C_n)^2
 *             + sum_n alpha^2 kappa_n / (2 c_s^2) sum_i w_i (C_n(x+c_i) - C_n(x))^2
 *             + (active == 1) beta (C1 - 1/2)^2 chi(x)  + fg C2 h(x) ]
 *     + (kcs == 0 ? -dP V : kcs/2 (V - V0)^2),  V = sum_x C2,  C3 = 1 - C1 - C2,
 * h(x) = the node's index along the last axis, chi(x) = 1 where the solid leaks
 * out of S (d_mask) or the fluid into it.  d_grad receives dE/dC2 (active = 2)
 * or dE/dC1 (active = 1).  d_terms (optional, 6 doubles): bulk, gradient,
 * confinement, constraint, gravity, V.  d_scratch: caller-owned device scratch
 * of at least dsm_fe_scratch_bytes() bytes.  Asynchronous on the stream. */
dsm_status dsm_fe_scratch_bytes(int lattice, int nx, int ny, int nz, size_t *bytes);
dsm_status dsm_fe_energy_grad(const dsm_params *p, const float *d_c1, const float *d_c2,
                              const unsigned char *d_mask, int active, double dP,
                              double kcs, double V0, double fg, double *d_energy,
                              float *d_grad, double *d_terms, void *d_scratch,
                              size_t scratch_bytes, void *cuda_stream);

/* Free energy of N = nfluid fluid components on a frozen solid (the N + 1
 * component model of Sec. II.A, which the paper states for any N and
 * demonstrates for N = 2).  Components: C_1 the solid (d_c1), the free fluids
 * C_2 .. C_N (d_c: N - 1 planes of nx*ny*nz floats, plane f holding
 * C_{2+f}), and C_{N+1} = 1 - C_1 - (C_2 + .. + C_N).  Each component k
 * carries kappa_k/2 C_k^2 (1 - C_k)^2 and the lattice-weighted gradient term
 * of dsm_fe_energy_grad with its own kappa_k (host array kappa, N + 1 values:
 * kappa_1 .. kappa_{N+1}), so any two components meet with tension
 * alpha (kappa_m + kappa_n) / 6.  Each free fluid f carries its own pressure
 * term -dP[f] V_f (kcs[f] == 0) or volume constraint kcs[f]/2 (V_f - V0[f])^2
 * (host arrays of N - 1 values; null for zeros), V_f = sum_x C_{2+f}.  No
 * gravity or confinement term.  From p: lattice, sizes, alpha and faces (the
 * tensions of p are not used).
 *   d_grad: N - 1 planes, dE/dC_{2+f} = d_{2+f} - d_{N+1} + the constraint's
 *   derivative, d_k = kappa_k b(C_k) - alpha^2 kappa_k L[C_k].
 *   d_terms (optional, 3 + N - 1 doubles): bulk, gradient, constraint, V_2..V_N.
 * 2 <= nfluid <= 4; every fluid kappa (k >= 2) > 0; kcs >= 0; otherwise
 * DSM_E_INVAL.  With N = 2 this is the stage-2 energy of dsm_fe_energy_grad
 * without gravity.  d_scratch: at least dsm_fe_multi_scratch_bytes() bytes,
 * 256-byte aligned.  Asynchronous on the stream. */
dsm_status dsm_fe_multi_scratch_bytes(int lattice, int nx, int ny, int nz, int nfluid,
                                      size_t *bytes);
dsm_status dsm_fe_energy_grad_multi(const dsm_params *p, int nfluid, const double *kappa,
                                    const float *d_c1, const float *d_c, const double *dP,
                                    const double *kcs, const double *V0, double *d_energy,
                                    float *d_grad, double *d_terms, void *d_scratch,
                                    size_t scratch_bytes, void *cuda_stream);

/* Allocation-free variant of dsm_fe_energy_grad, for callers that cannot
 * allocate device memory at all (a host program that links only this library
 * and has no CUDA allocator of its own, or an application whose device memory
 * is owned by an allocator that forbids side allocations).  The paper has no
 * counterpart: it is a service of this library.
 * Same arguments and results as dsm_fe_energy_grad minus the scratch buffer:
 * the reduction scratch is a fixed array of DSM_NOALLOC_SCRATCH_BYTES (64 KiB)
 * inside the library's device image, which every GPU that loads the library
 * holds until the process exits.  The energy kernel leaves at most one partial
 * sum per resident block (608), about 25 KB, whatever the lattice size, so every
 * lattice the library accepts fits; a lattice whose reduction did not fit would
 * be refused with DSM_E_WORKSPACE.  Invalid sizes are refused with DSM_E_INVAL
 * before any device work.  No device memory is allocated or freed by this call.
 * Each call looks up the array's device address in the current device's
 * context (cudaGetSymbolAddress, host-side; no allocation); the first call on
 * a device also loads the library's device image there, so make that first
 * call before any stream capture.  All calls on a device share the array: calls whose work
 * overlaps on the GPU (different streams, or several host threads) race on it
 * and must be serialised by the caller.  Every scratch word a call reads is
 * written earlier in the same call, so nothing needs clearing between calls. */
#define DSM_NOALLOC_SCRATCH_BYTES ((size_t)1 << 16)
dsm_status dsm_fe_energy_grad_noalloc(const dsm_params *p, const float *d_c1, const float *d_c2,
                                      const unsigned char *d_mask, int active, double dP,
                                      double kcs, double V0, double fg, double *d_energy,
                                      float *d_grad, double *d_terms, void *cuda_stream);

/* L-BFGS vector kernels for the energy minimiser (Sec. II.A cites L-BFGS,
 * Nocedal 1980; Liu & Nocedal 1989).  FP32 vectors, FP64 accumulation, results
 * written to device memory, deterministic (fixed reduction order).
 * d_scratch >= dsm_vec_scratch_bytes(n). */
dsm_status dsm_vec_scratch_bytes(long long n, size_t *bytes);
/* d_out[0] = sum_k x[k] * y[k] */
dsm_status dsm_vec_dot(long long n, const float *d_x, const float *d_y, double *d_out,
                       void *d_scratch, size_t scratch_bytes, void *cuda_stream);
/* y[k] += a * x[k] with a = sign * d_a[0] * (d_b ? d_b[0] : 1)  (device scalars) */
dsm_status dsm_vec_axpy_dev(long long n, double sign, const double *d_a, const double *d_b,
                            const float *d_x, float *d_y, void *cuda_stream);
/* y[k] = a * x[k] + b * y[k] with host scalars */
dsm_status dsm_vec_axpby(long long n, double a, const float *d_x, double b, float *d_y,
                         void *cuda_stream);
/* Two-loop recursion: d_r = -H g for the m stored pairs (newest last in the
 * ring order given by d_order[0..m-1], host array of slot indices, oldest
 * first).  d_S, d_Y: slot-major (slot*n + k).  d_rho: 1/(s.y) per slot (device
 * doubles).  d_gamma: device double, initial scaling s.y/y.y.  d_alpha: m device
 * doubles of scratch. */
dsm_status dsm_lbfgs_direction(long long n, int m, const int *order, const float *d_S,
                               const float *d_Y, const double *d_rho, const double *d_gamma,
                               const float *d_g, float *d_r, double *d_alpha,
                               void *d_scratch, size_t scratch_bytes, void *cuda_stream);

/* Batched vector kernels for the compact form of the L-BFGS matrix (Byrd,
 * Nocedal & Schnabel 1994: H = gamma I + [S gamma Y] M [S^T; gamma Y^T], the
 * same matrix as the two-loop recursion over the same pairs), which needs the
 * history only through two batched passes per iteration.
 * dsm_vec_dots: d_out[k] = V_k . x for k < nv, V_k = d_V + k * stride (FP32
 *   vectors of n elements), results as device doubles, each equal bitwise to a
 *   dsm_vec_dot of the same two vectors.  d_scratch >= dsm_vec_dots_scratch_bytes(n, nv).
 * dsm_vec_lincomb: y = cx x + sum_k coef[k] V_k (coef: host array of nv
 *   doubles, 0 <= nv <= 64, applied in FP32); y must not overlap x or any V_k.
 * Both asynchronous on the stream; DSM_E_INVAL for negative sizes, nv out of
 * range or a missing pointer. */
dsm_status dsm_vec_dots_scratch_bytes(long long n, int nv, size_t *bytes);
dsm_status dsm_vec_dots(long long n, int nv, const float *d_V, long long stride,
                        const float *d_x, double *d_out, void *d_scratch, size_t scratch_bytes,
                        void *cuda_stream);
dsm_status dsm_vec_lincomb(long long n, int nv, const float *d_V, long long stride,
                           const double *coef, const float *d_x, double cx, float *d_y,
                           void *cuda_stream);

/* The energy minimiser, native: L-BFGS over the active field (C2 for active = 2,
 * C1 for active = 1, the other field fixed in d_fixed) of the free energy of
 * dsm_fe_energy_grad with the same constraint arguments, from the start point
 * in d_x (FP32, nx*ny*nz, overwritten with the final point), until the rms
 * gradient sqrt(sum g^2 / N) < tol or max_iter iterations.  Sec. II.A cites
 * L-BFGS (Nocedal 1980; Liu & Nocedal 1989) with an rms-gradient stop; the
 * rest is this library's reading: m stored pairs (1 <= m <= 32), initial
 * matrix (s.y / y.y) I, pairs with s.y <= 1e-12 |s||y| dropped, a strong-Wolfe
 * line search (c1 = 1e-4, c2 = 0.9, cubic interpolation, at most 20 trials)
 * whose decrease test takes its derivative form when the energy change is
 * below 1e-6 |E| (FP32 noise), steepest descent after a non-descent direction,
 * and the direction from the compact form of the L-BFGS matrix (Byrd, Nocedal
 * & Schnabel 1994).  d_work: caller-owned device memory of at least
 * dsm_lbfgs_workspace_bytes(p, m), 256-byte aligned.  Runs on the stream and
 * returns when done.  The pair bookkeeping and the compact-form solve run on
 * the device; the host drives the line search and reads six doubles per trial
 * point (one read per iteration when the first trial is accepted).  At most 32
 * pairs (2m <= 64).  DSM_E_NONFINITE if the energy
 * or gradient turns non-finite.  dsm_lbfgs_compact is the host-only
 * compact-form solve, exposed for tests: for k pairs (oldest first),
 * SY[i*k+j] = s_i.y_j, YY[i*k+j] = y_i.y_j, a = S^T g, b = Y^T g, it returns the
 * coefficients of -H g = cx g + sum cs_i s_i + sum cy_i y_i. */
typedef struct dsm_lbfgs_info {
  long long iterations, evaluations;
  double energy, rms_grad;
  int converged;  /* 1 if the rms gradient fell below tol */
} dsm_lbfgs_info;
dsm_status dsm_lbfgs_workspace_bytes(const dsm_params *p, int m, size_t *bytes);
dsm_status dsm_lbfgs_minimize(const dsm_params *p, const float *d_fixed,
                              const unsigned char *d_mask, int active, double dP, double kcs,
                              double V0, double fg, float *d_x, int m, double tol,
                              long long max_iter, void *d_work, size_t work_bytes,
                              dsm_lbfgs_info *info, void *cuda_stream);
dsm_status dsm_lbfgs_compact(int k, const double *SY, const double *YY, const double *a,
                             const double *b, double gamma, double *cx, double *cs, double *cy);

/* The same L-BFGS over the N - 1 free fluid fields of dsm_fe_energy_grad_multi
 * together (d_x: N - 1 planes, overwritten with the final point; the solid
 * d_c1 fixed).  The rms gradient is taken over all planes.  d_work: at least
 * dsm_lbfgs_multi_workspace_bytes(p, nfluid, m) bytes, 256-byte aligned. */
dsm_status dsm_lbfgs_multi_workspace_bytes(const dsm_params *p, int nfluid, int m,
                                           size_t *bytes);
dsm_status dsm_lbfgs_minimize_multi(const dsm_params *p, int nfluid, const double *kappa,
                                    const float *d_c1, const double *dP, const double *kcs,
                                    const double *V0, float *d_x, int m, double tol,
                                    long long max_iter, void *d_work, size_t work_bytes,
                                    dsm_lbfgs_info *info, void *cuda_stream);

/* Batched step: advance handle i by nsteps[i] stage-2 steps, all handles in
 * ONE persistent cooperative launch.  Resident blocks walk a work list of
 * (lattice, 32-node-wide brick) pairs of every lattice: per step a moments
 * phase and a fused phase, each followed by a grid-wide barrier whose waits are
 * bounded (a barrier that does not complete within a few seconds latches
 * DSM_E_TIMEOUT in every handle of the batch, reported by the next
 * dsm_get_observables).  For many small lattices this replaces two launches per
 * lattice per step by one launch per call.  Each lattice's result equals its
 * solo dsm_step result bitwise (same per-node arithmetic).
 * Requirements: n >= 1; every handle with fluid set and no latched error; all
 * share the lattice kind, the precision, the stream, and whether rho2 != rho3;
 * otherwise DSM_E_INVAL.  d_scratch: caller-owned device memory of at least
 * dsm_batch_scratch_bytes(hs, n) bytes, 256-byte aligned (work list, per-lattice
 * arguments, barrier words); DSM_E_WORKSPACE if short.  The call waits for its
 * small host-to-device copies of the work list, then returns with the launch
 * queued on the stream. */
dsm_status dsm_batch_scratch_bytes(dsm_lattice *const *hs, int n, size_t *bytes);
dsm_status dsm_batch_step(dsm_lattice *const *hs, int n, const long long *nsteps, void *d_scratch,
                          size_t scratch_bytes);

/* Release the handle (host memory only; the workspace stays the caller's). */
/* Polls a bounded device wait makes before it gives up: the grid barriers of
 * dsm_batch_step poll a flag that the last block to arrive sets, and after
 * this many polls (default 0: 2e7 polls, a few seconds) a block stops waiting,
 * latches DSM_E_TIMEOUT in every lattice of the launch and returns, so the
 * kernel always ends.  The next synchronising call (dsm_get_observables)
 * reports DSM_E_TIMEOUT and the handles stay latched (DSM_E_STATE) until
 * dsm_set_state, dsm_set_populations or dsm_set_fluid.  A small limit makes
 * early blocks give up and exercises that path.  Process-wide; not
 * thread-safe against concurrent dsm_batch_step calls. */
dsm_status dsm_set_wait_limit(unsigned long long polls);

dsm_status dsm_destroy(dsm_lattice *h);

/* ---- N fluid components, lattice Boltzmann ------------------------------
 * The stage-2 step for N = nfluid fluids (2 <= N <= 4) on a frozen diffuse
 * solid: the N + 1-component model of Sec. II.B, which the paper states for
 * any N and demonstrates for N = 2.  Fluids C_2 .. C_N are free, each with its
 * own Cahn-Hilliard populations; C_{N+1} = 1 - C_1 - (C_2 + .. + C_N).
 * Host arrays: kappa (N + 1 values, kappa_1 .. kappa_{N+1}: the tension of
 * components m, n is alpha (kappa_m + kappa_n) / 6), rho and tau (N values,
 * fluids 2 .. N + 1).  From p: lattice, sizes, precision (DSM_F64 or DSM_F32;
 * others DSM_E_UNSUPPORTED), alpha, alpha_s, tau_g, body_force (on fluid 2),
 * faces.  Population form; one step = the moments pass and the fused pass:
 *   mu_f = d_f - d_{N+1},  d_k = kappa_k b(C_k) - alpha^2 kappa_k L[C_k];
 *   F = sum_f mu_f G[C_f] + C_2 b;
 *   rho = rho_{N+1} + sum_f (rho_f - rho_{N+1}) phi_f, phi_f = C_f / (1 - C_1)
 *   clamped to [0, 1]; tau = the tau of the locally largest fluid (ties to the
 *   later fluid); interpolated bounce-back and the face rules as for N = 2.
 * With tau_g = 1 and every face periodic each g_f is held as g_eq (the
 * post-collision g_f is g_eq, fixed by A_f = mu_f - 3/2 C_f u.u, C_f and u):
 * the fused pass stores A_f and u instead of Q populations per fluid and the
 * moments pass rebuilds C_f from them, as dsm_set_g_storage's DSM_G_AUTO does
 * for two fluids.  Otherwise g_f is stored as populations.  With N = 2 this is
 * dsm_step in the same storage form.  The workspace (at least
 * dsm_ml_workspace_bytes, 256-byte aligned) is the caller's.  dsm_ml_set_solid
 * takes a signed distance (kind 0) or C1 itself (kind 1); dsm_ml_set_fluids
 * the free fluids (N - 1 planes of nx*ny*nz reals) and writes the rest state.
 * dsm_ml_get_field: DSM_FIELD_C2 with index f gives C_{2+f} (index N - 1: the
 * dependent fluid), DSM_FIELD_MU with index f gives mu_{2+f}, DSM_FIELD_C1,
 * UX, UY, UZ, PT, RHO, TAU as for dsm_get_field; DSM_FIELD_C3 is DSM_E_INVAL.
 * dsm_ml_get_populations: f (Q planes) and g (N - 1 blocks of Q planes), dense
 * nx*ny*nz rows (held as g_eq: rebuilt from (A_f, C_f, u)).  The fused pass
 * latches a non-finite state in the workspace; dsm_ml_check synchronises the
 * stream and returns DSM_E_NONFINITE once it is latched, DSM_E_TIMEOUT for a
 * timed-out wait of the one-pass step, DSM_E_BOUNDS for an index fault caught
 * by the checked build (dsm_ml_set_fluids clears all three). */
typedef struct dsm_mlattice dsm_mlattice;
dsm_status dsm_ml_workspace_bytes(const dsm_params *p, int nfluid, size_t *bytes);
dsm_status dsm_ml_create(const dsm_params *p, int nfluid, const double *kappa,
                         const double *rho, const double *tau, void *d_workspace,
                         size_t bytes, void *cuda_stream, dsm_mlattice **out);
dsm_status dsm_ml_set_solid(dsm_mlattice *h, const void *d_field, int kind);
dsm_status dsm_ml_set_fluids(dsm_mlattice *h, const void *d_c);
dsm_status dsm_ml_step(dsm_mlattice *h, long long nsteps);
dsm_status dsm_ml_get_field(dsm_mlattice *h, int field, int index, void *d_dst);
dsm_status dsm_ml_get_populations(dsm_mlattice *h, void *d_f, void *d_g);
dsm_status dsm_ml_check(dsm_mlattice *h);
dsm_status dsm_ml_destroy(dsm_mlattice *h);

/* How dsm_ml_step advances an N-fluid lattice, as dsm_set_step_form does for
 * two fluids.  For D3Q19 lattices that hold every g_f as g_eq (tau_g = 1,
 * periodic faces) with nx >= 32 and ny >= 8,
 * DSM_STEP_AUTO runs each step as ONE pass: blocks march 32 x 8 tiles up runs
 * of z planes, stage the previous collision's (A_f, C_f) of every free fluid,
 * u and C1 into shared memory by tensor-memory-accelerator copies, rebuild
 * every C_f of the step on the tile and a one-node halo, and run the fused
 * pass from there.  The same step up to FP contraction order; the state then
 * lives in padded buffers of the workspace (per padded node, (nx + 8 rounded
 * up to a multiple of 4)(ny + 4)
 * nz of them, two buffers of 5 + 2 (N - 2) reals, and C1; included in
 * dsm_ml_workspace_bytes) and is converted back before dsm_ml_get_field or
 * dsm_ml_get_populations reads it.  A staged plane that never arrives (a
 * bounded wait of about two seconds) latches DSM_E_TIMEOUT, which
 * dsm_ml_check returns.  DSM_STEP_TWO_PASS always runs the two passes.  zrun:
 * z planes per block, 0 = chosen from the lattice and the GPU.  DSM_E_INVAL
 * for an unknown form or zrun < 0. */
dsm_status dsm_ml_set_step_form(dsm_mlattice *h, int form, int zrun);

/* Whether dsm_ml_step runs the one-pass step (*single_pass = 1) and with how
 * many z planes per block (*zrun; 0 for the two-pass step).  Either pointer
 * may be NULL. */
dsm_status dsm_ml_step_info(dsm_mlattice *h, int *single_pass, int *zrun);

#ifdef __cplusplus
}
#endif
#endif /* DSM_H */
