/*
 * lbm.h -- C ABI of the B300 D2Q37 thermal lattice Boltzmann step.
 *
 * Method: Ripesi, Biferale, Schifano & Tripiccione, "Evolution of a double-front
 * Rayleigh-Taylor system using a GPU-based high resolution thermal Lattice-Boltzmann
 * model", Phys. Rev. E 89, 043022 (2014).  One time step is the lattice BGK update of
 * Sec. III.A Eq. (LBE): pull-propagate of the 37 populations with periodic x
 * (Sec. III.B, steps pbc and propagate), the top/bottom wall rule on rows 0..2 and
 * Lz-3..Lz-1 (Sec. III.B, step bc) and the collide with the force-shifted equilibrium
 * f^eq[rho, u + tau g, T + tau (1 - tau) g^2 / D] (Sec. III.A).
 *
 * Conventions shared by every entry point
 *   - Lattice Lx x Lz sites; x periodic, z bounded by walls at z = -1/2 and Lz - 1/2.
 *     Lx >= 1, Lz >= 6 and 37 * Lx * Lz < 2^31.
 *   - Units: dt = 1, reference temperature 1, xi_l = r c_l (r ~ 1.1969, Sec. III.A),
 *     gravity vector (0, -g) with g >= 0 (z points up, Sec. II Eq. (NS)).
 *   - Population storage is structure-of-arrays, column-major (Sec. III.B):
 *     element (l, x, z) at ((l * Lx) + x) * Lz + z, z fastest.  The canonical velocity
 *     order is l = 0 for (0,0), then the shells |c|^2 = 1,2,4,5,8,9,10, each sorted by
 *     the polar angle atan2(c_z, c_x) in [0, 2 pi).
 *   - Wall rule (Sec. III.B names the rows, not the rule; this library's reading):
 *     half-way bounce-back on the same column: a pull source row z - c_z below 0 is
 *     replaced by population opp(l) at row c_z - 1 - z, one at or above Lz by opp(l) at
 *     row 2 Lz - 1 - z + c_z.  Propagate + bc is then a permutation of (l, x, z).
 *   - Device pointers are CUDA device addresses on the context's device; host
 *     pointers are ordinary host memory.  Buffers passed in are BORROWED: the caller
 *     (e.g. PyTorch) owns them and must keep them alive until lbm_destroy.
 *   - Calls are asynchronous on the context's stream unless stated.  Kernel-side
 *     errors surface at the next synchronising call (lbm_sync, or any call that
 *     copies to the host).
 *   - Every int-returning call returns LBM_OK (0) or a negative LBM_E* code; the
 *     message of the last failure on the calling thread is lbm_last_error().
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,     /* invalid argument (shape, pointer, size, precision)          */
    LBM_ECUDA = -2,      /* a CUDA runtime call failed                                  */
    LBM_ENOMEM = -3,     /* a context-private allocation failed                         */
    LBM_ETIMEOUT = -4,   /* a bounded device-side wait gave up                          */
    LBM_ENUMERIC = -5,   /* non-finite values detected                                  */
    LBM_ESTATE = -6      /* call not valid in the context's current state              */
};

/* Population storage and collide arithmetic.
 *   LBM_F64     IEEE binary64 storage, collide in native FP64 arithmetic.
 *   LBM_F32     FP32 storage, FP32 collide arithmetic (compensated moment sums; the
 *               collide update is repaired to conserve mass, momentum + rho g and
 *               internal energy).
 *   LBM_F32_DEV FP32 storage of the deviation d = f - fref(l, z) from a per-row
 *               reference, fref = f^eq(rho0(z), gvec/2, T0(z)) at the horizontal means
 *               rho0, T0 of the rows of the last lbm_init_layers state (of a uniform
 *               rho = T = 1 state before it), kept by the context in FP64; FP32 collide
 *               arithmetic on deviations only (the reference's moments per row from
 *               FP64 tables).  The step, the state copies and the diagnostics take it;
 *               thermal walls, the push form, lbm_propagate, the slabs, the ensembles and
 *               every adjoint entry point return LBM_ESTATE for it, lbm_step_host
 *               LBM_EINVAL (it takes FP64 storage).  The diagnostics work on an FP64 copy
 *               of the state in a temporary device buffer (37*Lx*Lz doubles).
 *   LBM_F64_FF  IEEE binary64 storage; moments summed in 64-bit integers, the rest of
 *               the collide in float-float arithmetic (pairs of FP32 carrying a ~48-bit
 *               significand) on the FP32 and integer pipes, one FP64 FMA per population
 *               for the relaxation; same storage and bytes as LBM_F64, results equal to
 *               it to ~1e-14 per step.                                                 */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F32_DEV = 2, LBM_F64_FF = 3 } lbm_prec;

typedef struct lbm_ctx lbm_ctx;   /* opaque */

/* Three-layer initial state of Sec. I (Eq. (seteq), pressure continuity, Fig. 1
 * caption).  Heights are in sites with row k at height k + 1/2; interfaces are
 *   z_lo(x) = z_lo + sum_k amp_lo[k-1] cos(2 pi k x / Lx + phase_lo[k-1]), k = 1..n_modes,
 * and z_hi(x) likewise.  Pressure is isothermal-hydrostatic in each layer and
 * continuous across both interfaces, p = rho_ref T_d exp(-g r z / T_d) below z_lo(x);
 * T(x,z) = T_u + (T_m-T_u)(1 - tanh((z - z_hi)/w))/2 + (T_d-T_m)(1 - tanh((z - z_lo)/w))/2,
 * rho = p / T, populations f^eq(rho, u = (0, -g/2), T) (renormalised velocity zero).
 * The four mode arrays are host arrays of n_modes doubles owned by the caller and
 * read during the call only.                                                          */
typedef struct {
    double T_u, T_m, T_d;          /* top, middle, bottom temperatures (> 0)            */
    double z_lo, z_hi;             /* unperturbed interface heights in sites              */
    double rho_ref;                /* density at the bottom wall in the bottom layer      */
    double tanh_w;                 /* interface half-width w in sites (> 0)               */
    int    n_modes;                /* K >= 0                                              */
    const double *amp_lo, *phase_lo, *amp_hi, *phase_hi;
} lbm_layers_desc;

/* Create a context for an Lx x Lz lattice with relaxation time tau > 0.5 and gravity
 * g >= 0 (Sec. III.A).  buf0 and buf1 are 16-byte aligned device buffers on one device
 * of at least 37*Lx*Lz*(8 for LBM_F64 / LBM_F64_FF, 4 for LBM_F32 / LBM_F32_DEV) bytes
 * each, `bytes` the size of each; they hold the two lattice copies (Sec. III.B: read
 * one, write the other, swap).  The state starts in buf0.  cuda_stream is a
 * cudaStream_t (NULL: the legacy default stream).  The context allocates only small
 * private scratch (reduction partials, mode parameters, an error word; for LBM_F32_DEV
 * also the reference tables, 37*Lz doubles and 26*Lz floats).  On failure *out is NULL.  */
int lbm_create(lbm_ctx **out, int Lx, int Lz, int prec, double tau, double g,
               void *buf0, void *buf1, size_t bytes, void *cuda_stream);

/* Release the context's private scratch; the borrowed buffers are untouched.
 * Synchronises the stream first.  NULL is accepted.                                   */
int lbm_destroy(lbm_ctx *c);

/* Write the three-layer initial state (see lbm_layers_desc) into the current lattice
 * copy.  LBM_EINVAL for non-positive temperatures, width or rho_ref, n_modes < 0, or
 * NULL mode arrays with n_modes > 0.                                                  */
int lbm_init_layers(lbm_ctx *c, const lbm_layers_desc *d);

/* Advance nsteps >= 0 time steps (propagate + bc + collide, Sec. III.A-B), one fused
 * kernel launch per step, ping-ponging between the two buffers.  Asynchronous.       */
int lbm_step(lbm_ctx *c, int nsteps);

/* Wall rule of lbm_step and lbm_step_host (Sec. III.B names only the bc rows 0..2 and
 * Lz-3..Lz-1).  thermal = 0 (the default): adiabatic no-slip half-way bounce-back.
 * thermal = 1: isothermal walls at T_bottom (z = -1/2) and T_top (z = Lz - 1/2): a
 * population whose pull source row lies beyond a wall takes the value of one of three
 * ghost rows holding f^eq(rho_w(x), 0, T_w) (the unshifted equilibrium at rest), with
 * the ghost density of each column set so that the mass the step moves into the ghost
 * rows of that column equals the mass the ghost rows send into the lattice (total mass
 * is conserved).  With thermal walls, lbm_step_push, the slab decomposition, the
 * ensembles, the moment records and the adjoint of LBM_F64 contexts return LBM_ESTATE
 * (they implement the bounce-back rule only); the adjoint of LBM_F64_FF contexts follows
 * the thermal rule.  LBM_EINVAL for thermal outside {0, 1} or non-positive / non-finite wall
 * temperatures.  Host only; takes effect from the next step.                          */
int lbm_set_walls(lbm_ctx *c, int thermal, double T_bottom, double T_top);

/* Push form of the step (Sec. III.B compares "push" and "pull"; lbm_step is the pull form,
 * whose stored state is post-collision, f <- C(P f)).  lbm_step_push advances a state
 * stored post-propagation (pre-collision), g <- P(C g): every site reads its own
 * populations (aligned) and writes each result at the site it moves to (misaligned), the
 * wall rule mirrored.  Same collide arithmetic as lbm_step in every precision.
 * Asynchronous.                                                                       */
int lbm_step_push(lbm_ctx *c, int nsteps);

/* One propagate + bc without collide, f <- P f (the pull gather).  It maps a pull-form
 * state to the matching push-form one: push steps from P f equal P applied to the pull
 * steps from f.  Asynchronous.                                                        */
int lbm_propagate(lbm_ctx *c);

/* Steps through caller-owned device buffers: states[j + 1] = step(states[j]) for
 * j = 0 .. n - 2 (n >= 0 pointers, each 37*Lx*Lz populations in the context's storage
 * precision and layout), with the context's tau, g and wall rule; the context's own
 * state is neither read nor changed.  Consecutive buffers must differ.  Serves the
 * recomputation of a checkpoint segment before its adjoint without copies.  Asynchronous. */
int lbm_step_chain(lbm_ctx *c, void *const *states, int n);

/* Device address of the buffer holding the current state (buf0 or buf1); NULL for a
 * NULL context.                                                                       */
void *lbm_current(lbm_ctx *c);

/* Copy the current state out / in as canonical FP64 f[l][x][z] (37*Lx*Lz doubles).
 * on_device = 1: `f` is a device pointer (stream-ordered, asynchronous); 0: a host
 * pointer (the call synchronises).  FP32 storage is converted; LBM_F32_DEV copies out
 * f_ref(l, z) + d in FP64 and stores (float)(f - f_ref(l, z)) on the way in.              */
int lbm_get_populations(lbm_ctx *c, double *f, int on_device);
int lbm_set_populations(lbm_ctx *c, const double *f, int on_device);

/* Host-buffer stepping, streamed: for t = 0..n-1 the state host_in[t] (canonical FP64
 * f[l][x][z], 37*Lx*Lz doubles) is copied in, advanced one step (lbm_step), and the result
 * copied out to host_out[t].  The copy out of step t-1 and the copy in of step t run
 * concurrently on two copy streams (one per direction of the host link), each step on the
 * context's stream once both are done with its buffers; with pinned host buffers the
 * transfer time per step is that of one direction.  Uses the context's two buffers (the
 * device holds the last step's output afterwards).  FP64 storage (LBM_F64, LBM_F64_FF)
 * only; LBM_EINVAL otherwise or for NULL buffers.  Synchronises before returning.       */
int lbm_step_host(lbm_ctx *c, const double *const *host_in, double *const *host_out, int n);

/* Per-site fields of the current (post-collision) state, Sec. III.A: rho, u, T with
 * D rho T = sum |xi - u|^2 f.  renormalised = 1 returns u^H = u - gvec/2 (the paper's
 * u + dt g/2 of the pre-collision state) and T^H = T + g^2/(4 D).  Each output is an
 * [Lx][Lz] array (z fastest) or NULL to skip; on_device as for lbm_get_populations.   */
int lbm_moments(lbm_ctx *c, double *rho, double *ux, double *uz, double *T,
                int renormalised, int on_device);

/* Horizontal mean T(z) = (1/Lx) sum_x T(x, z) of the raw temperature (Sec. IV), Lz
 * doubles, reduced in FP64 on the device in a fixed order.  on_device as above.      */
int lbm_row_mean_T(lbm_ctx *c, double *Tbar, int on_device);

/* Threshold mixing widths of the two fronts from the current state (Sec. IV: the
 * region where the mean profile lies between 5% and 95% of each layer jump).  Upper
 * front: b = (Tbar - T_u)/(T_m - T_u) scanned top-down, first crossing of 0.05 then of
 * 0.95; lower front: b = (Tbar - T_m)/(T_d - T_m) scanned bottom-up, 0.95 then 0.05;
 * crossings linearly interpolated between consecutive rows.  out[0] = L_u, out[1] =
 * L_d in sites (host).  If dL_dTbar is not NULL it receives d(L_u + L_d)/dTbar(z)
 * (host array of Lz doubles).  Synchronises.  LBM_EINVAL when a crossing is missing
 * or the temperatures are not ordered T_u < T_m < T_d.                                */
int lbm_widths(lbm_ctx *c, double T_u, double T_m, double T_d, double out[2], double *dL_dTbar);

/* Tent-map mixing widths of the two fronts, Eq. (3L) of Sec. IV:
 *   L_u = sum_z Theta[(Tbar(z) - T_u) / (T_m - T_u)],  L_d = sum_z Theta[(Tbar(z) - T_m) / (T_d - T_m)],
 * with Theta[b] = 2 b on (0, 1/2), 2 (1 - b) on [1/2, 1) and 0 elsewhere, Tbar the horizontal
 * mean of the raw T (lbm_row_mean_T), the integral over z taken as the sum over rows (in
 * sites).  For a single front pass a virtual T_m between T_u and T_d.  Host out[2] =
 * {L_u, L_d}.  Synchronises.  LBM_EINVAL unless T_u < T_m < T_d.                       */
int lbm_tent_widths(lbm_ctx *c, double T_u, double T_m, double T_d, double out[2]);

/* Per-row statistics over x of the current state (the fluctuation profiles of Sec. IV):
 * mean and rms fluctuation sqrt(<(q - <q>_x)^2>_x) of q = T (raw) and of q = E_k, the
 * kinetic energy per unit mass |u^H|^2 / 2 with u^H the renormalised velocity.  Two
 * passes (means, then squared deviations), FP64, fixed summation order.  Each output is
 * an array of Lz doubles or NULL to skip; on_device as for lbm_get_populations.        */
int lbm_row_stats(lbm_ctx *c, double *T_mean, double *T_rms, double *Ek_mean, double *Ek_rms, int on_device);

/* Total mass sum f and energy sum |xi|^2 f / 2 of the current state, reduced in FP64
 * in a fixed order (host out[2]).  Synchronises; LBM_ENUMERIC if either is not
 * finite.                                                                             */
int lbm_global_sums(lbm_ctx *c, double out[2]);

/* Adjoint of one step.  With f_{t+1} = C(P f_t), P the propagate+bc permutation and C the
 * pointwise collide (Eq. (LBE) with the shifted equilibrium of Sec. III.A):
 *   lam_out = P^T J_C(P f_t)^T lam_next.
 * f_t, lam_next, lam_out: device arrays of 37*Lx*Lz populations in the context's storage
 * precision and layout (double for LBM_F64 / LBM_F64_FF, float for LBM_F32); lam_out must
 * not alias the other two.  LBM_F64 evaluates the Jacobian product in native FP64, LBM_F32
 * in FP32 (the gradient of an FP32 run to FP32 rounding); LBM_F64_FF in float-float on the FP32 pipes with one FP64 FMA per
 * population, scaled per site by the largest exponent among its 37 lam_next values
 * (entries more than 2^74 below that maximum count as 0 in the collide term; results
 * agree with the native form to ~1e-15 of the site's largest |lam_next|).  Both assume
 * |u| well below 0.3 and finite inputs.  With thermal walls (lbm_set_walls; LBM_F64_FF
 * only) propagate + bc is linear rather than a permutation: lam_out is its transpose, a
 * population that leaves through a wall receiving the sum, over the destinations that pull
 * from its ghost column, of their mu times f^eq_l(1, 0, T_w) / in_w; a second launch forms
 * those sums in a fixed order, and the first call allocates 6*37*Lx doubles of scratch
 * (LBM_ENOMEM if that fails).  Asynchronous.                                            */
int lbm_adjoint_step(lbm_ctx *c, const void *f_t, const void *lam_next, void *lam_out);

/* n adjoint steps in one call: with lam_a holding lam_n on entry, applies lbm_adjoint_step
 * for t = n - 1 down to 0 with f_t = states[t], ping-ponging between lam_a and lam_b;
 * *out_index = 0 if lam_0 ends in lam_a, 1 if in lam_b.  The states (device, the context's
 * storage precision and layout) must not alias lam_a or lam_b.  Same precision and wall conditions as lbm_adjoint_step.
 * Asynchronous.                                                                         */
int lbm_adjoint_chain(lbm_ctx *c, const void *const *states, int n, void *lam_a, void *lam_b,
                      int *out_index);

/* The adjoint of a step needs f_t only through the fixed-point moments (rho, J = sum c g,
 * E = sum |c|^2 g, unit 2^-60, int64) of the pulled g = P f_t at each site, which the step
 * itself forms.  lbm_record_moments runs n steps from f0 (device, FP64 layout, unchanged),
 * alternating the outputs between work_a and work_b (the state after step j is in work_a for
 * even j, work_b for odd j), and writes the moments of step j to moments[j]: 4*Lx*Lz int64,
 * planes R, Jx, Jz, E of Lx*Lz sites each (site x*Lz + z).  lbm_adjoint_chain_moments is
 * lbm_adjoint_chain with f_t replaced by such records (moments[t] for step t), bit for bit
 * the same result, reading 32 instead of 296 bytes of f_t per site.  LBM_F64_FF contexts
 * with bounce-back walls only (LBM_ESTATE otherwise); f0, work_a, work_b distinct.
 * Asynchronous.                                                                         */
int lbm_record_moments(lbm_ctx *c, const double *f0, int n, double *work_a, double *work_b,
                       int64_t *const *moments);
int lbm_adjoint_chain_moments(lbm_ctx *c, const int64_t *const *moments, int n, double *lam_a,
                              double *lam_b, int *out_index);

/* Adjoint of the width readout: lam(l,x,z) = dL_dTbar[z] / Lx * dT(x,z)/df_l with
 * dT/df_l = (|xi_l - u|^2 - D T) / (D rho) at the state f (device).  f and lam_out: 37*Lx*Lz
 * populations in the context's storage precision (FP64 arithmetic); dL_dTbar is a host array
 * of Lz doubles.  Synchronises.                                                          */
int lbm_loss_adjoint(lbm_ctx *c, const void *f, const double *dL_dTbar, void *lam_out);

/* Adjoint of lbm_init_layers with respect to the mode amplitudes: given lam0 = dL/df_0
 * (device, the context's storage precision and layout) returns dL/damp_lo[k] and
 * dL/damp_hi[k] in the host arrays dA_lo, dA_hi (n_modes each).  Synchronises.          */
int lbm_init_adjoint(lbm_ctx *c, const lbm_layers_desc *d, const void *lam0,
                     double *dA_lo, double *dA_hi);

/* lbm_init_adjoint plus, when dph_lo and dph_hi are given (both or neither), the gradient with
 * respect to the mode phases: the interfaces z(x) = z0 + sum_k A_k cos(2 pi k x / Lx + phi_k)
 * (Sec. I) give dL/dphi_k = -A_k sum_x dL/dz(x) sin(2 pi k x / Lx + phi_k).  Host arrays of
 * n_modes doubles.  Synchronises.                                                         */
int lbm_init_adjoint_full(lbm_ctx *c, const lbm_layers_desc *d, const void *lam0,
                          double *dA_lo, double *dA_hi, double *dph_lo, double *dph_hi);

/* Wait for all work queued by this context; reports deferred kernel-side errors.     */
int lbm_sync(lbm_ctx *c);

/* Lattice constants of the library's own quadrature solve (host only, no GPU needed):
 * c (37 x 2 ints, canonical order), w (37 doubles), r.  Any pointer may be NULL.      */
int lbm_lattice(int *c, double *w, double *r);

/* ---------------------------------------------------------------------------------
 * Ensembles: independent lattices (the paper's N_conf realisations of one setup, Table
 * II) advanced together.  An ensemble groups existing contexts that share device,
 * precision (LBM_F64_FF or LBM_F32), tau, g and stream; each keeps its own buffers and
 * sizes.  Results are identical to stepping each context alone.
 * ------------------------------------------------------------------------------- */
typedef struct lbm_ensemble lbm_ensemble;

/* Group n contexts (borrowed; they must outlive the ensemble).                        */
int lbm_ensemble_create(lbm_ensemble **out, int n, lbm_ctx *const *ctxs);
int lbm_ensemble_destroy(lbm_ensemble *e);

/* Launch shape: mode 0 = one launch per step over the tiles of all lattices; mode 1 =
 * one persistent cooperative launch for all steps, CTAs taking work items (a step and 8
 * consecutive tiles of one lattice) from a step-major queue with a per-lattice step
 * barrier (an item of step s waits until all tiles of step s-1 of its lattice are done).
 * tile_z: threads (rows) per tile, 64, 128 or 256.  ctas_per_sm: persistent CTAs per SM
 * (0: as many as fit).                                                                */
int lbm_ensemble_config(lbm_ensemble *e, int mode, int tile_z, int ctas_per_sm);

/* Autotuner: times `steps` steps (after a warm-up of the same length) for every mode,
 * tile_z and CTA count, keeps the fastest and reports it (any output may be NULL;
 * best_ms per step).  The trial runs advance the lattices' state.                     */
int lbm_ensemble_tune(lbm_ensemble *e, int steps, double *best_ms, int *best_mode, int *best_tile_z,
                      int *best_ctas_per_sm);

/* Advance every lattice by nsteps (asynchronous on the shared stream).                */
int lbm_ensemble_step(lbm_ensemble *e, int nsteps);

/* Capture one lbm_ensemble_step(e, nsteps) into a CUDA graph (the stream must not be the
 * legacy default stream); lbm_ensemble_graph_launch replays it.  A replay requires every
 * lattice to be in the buffer it was in at capture (always true for even nsteps).      */
int lbm_ensemble_capture(lbm_ensemble *e, int nsteps);
int lbm_ensemble_graph_launch(lbm_ensemble *e);

/* Wait for the stream; LBM_ETIMEOUT if a persistent launch's bounded barrier wait ran
 * out (the error word is then cleared).                                                */
int lbm_ensemble_sync(lbm_ensemble *e);

/* Bounded-wait parameters of the persistent launch: the cycle budget of one barrier wait
 * (default 4e9, about 2 s) and an extra count added to every barrier target (default 0;
 * a positive value makes every wait run out, for testing the timeout path).            */
int lbm_ensemble_set_wait(lbm_ensemble *e, long long spin_limit_cycles, unsigned int extra_wait);

/* Horizontal mean T(z) of an FP64 population array, allocating nothing.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory when they need the diagnostic -- a plugin whose device memory
 * is all handed to it by a host application, code whose memory belongs to a pool or
 * budget it does not control, or a latency-critical loop where cudaMalloc's implicit
 * device synchronisation is not acceptable -- and so cannot create an lbm_ctx
 * (lbm_create allocates scratch) or let lbm_row_mean_T grow its reduction buffer.
 * f: device array of 37*Lx*Lz doubles in the storage layout; Tbar: device array of Lz
 * doubles (output); both on the current device; cuda_stream: cudaStream_t or NULL.
 * The two-stage reduction of lbm_row_mean_T runs with its partial sums in one static
 * device array of 2^20 doubles (8 MiB) that every GPU loading the library keeps until
 * process exit; Lz above 1,048,576 is rejected with LBM_EINVAL.  The partial sums are
 * fully rewritten by every call, so nothing needs clearing; but all calls on a device
 * share that array, so calls that may overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The first call on a device does
 * a one-time set-up (lattice constants, scratch address) with host synchronisation, so
 * make it before any stream capture.  The library keeps that set-up (here and for every
 * context) for the life of the process: resetting a device's primary context
 * (cudaDeviceReset) while the library is loaded is not supported.  Calls no
 * cudaMalloc/cudaFree.  Asynchronous.                                                  */
int lbm_row_mean_T_noalloc(const double *f, int Lx, int Lz, double *Tbar, void *cuda_stream);

/* ---------------------------------------------------------------------------------
 * x-slab decomposition (Sec. III.B: the lattice split along x into slabs of Lx/nslab
 * columns, each with H_x = 3 halo columns per side refreshed from its neighbours before
 * every step), run on the device of one context.  The slabs live in library-owned buffers
 * (2 copies of nslab * 37 * (Lx/nslab + 6) * Lz populations).  Results equal lbm_step's
 * bit for bit.
 * ------------------------------------------------------------------------------- */
typedef struct lbm_slabs lbm_slabs;   /* opaque */

/* Slabs for the lattice of c.  LBM_EINVAL unless nslab divides Lx with at least 3
 * columns per slab; LBM_ENOMEM if the buffers cannot be allocated.                    */
int lbm_slabs_create(lbm_slabs **out, lbm_ctx *c, int nslab);
int lbm_slabs_destroy(lbm_slabs *s);

/* Copy the context's current state into the slabs (asynchronous, c's stream).         */
int lbm_slabs_scatter(lbm_slabs *s);

/* nsteps steps of every slab: halo exchange by device copies, then the step kernel on
 * each slab's own columns.  overlap = 1 (and slabs wider than 6 columns): the columns that
 * need no halo run on a second stream while the exchange and the edge columns run on c's
 * stream, the paper's overlap of communication with the bulk update; 0: exchange, then
 * whole slabs, all on c's stream.  Asynchronous with respect to the host.             */
int lbm_slabs_step(lbm_slabs *s, int nsteps, int overlap);

/* Copy the slabs' state back into the context's current buffer; synchronises.       */
int lbm_slabs_gather(lbm_slabs *s);

/* Bounds-checked builds (liblbm_checked.so, compiled with -DLBM_BOUNDS_CHECK): *out = the
 * number of out-of-range population indices the kernels met on the current device since the
 * last call (each one was redirected to element 0 instead of being used); the count is reset.
 * Synchronises the device.  Other builds: LBM_ESTATE.  The paper has no counterpart.     */
int lbm_test_oob_count(unsigned int *out);

/* Test hook for the error paths: the n-th next device allocation made by the library
 * (n = 0: the next one) is refused as if the device were out of memory; the caller
 * reports LBM_ENOMEM.  One refusal per call of this function; n < 0 cancels a pending one.
 * The paper has no counterpart.                                                       */
int lbm_test_fail_alloc(int n);

/* Test hook for the packed float-float arithmetic of the step and adjoint kernels (two values
 * in the lanes of B300's packed FP32 registers): runs n seeded pairs of operands through every
 * packed operation and its scalar form on the current device and stores in *mismatches the
 * number of result words whose bits differ (0 when each lane reproduces the scalar form).
 * Synchronises the device.  LBM_EINVAL for n < 1 or a NULL pointer.  The paper has no
 * counterpart.                                                                          */
int lbm_test_packed_ff(int n, unsigned long long seed, unsigned long long *mismatches);

/* Throughput of the current device's FP64 pipe, the second roof of the FP64-storage steps
 * (their FP64 instructions per site against it, beside their DRAM bytes per site against the
 * HBM bandwidth): two launches of 8 blocks of 256 threads per SM, each thread running 8
 * independent chains of iters FMAs; the second launch is timed with CUDA events on the
 * legacy default stream.  *fma_per_s = thread-level FP64 FMAs per second (a pure FP64
 * stream: kernels that mix FP64 with other work can run the pipe about 5% faster).  Synchronises
 * the device.  LBM_EINVAL for iters outside 1 .. 2^18 or a NULL pointer.  The paper has no
 * counterpart.                                                                          */
int lbm_probe_fp64_rate(int iters, double *fma_per_s);

/* Message of the last failed call on this thread ("" if none).                        */
const char *lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
