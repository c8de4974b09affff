/*
 * lbm.h -- C ABI of the GB300 (sm_103a) D3Q19 lattice Boltzmann library.
 *
 * The library implements the fused stream + collide time step of the D3Q19
 * lattice Boltzmann method with a per-run choice between the standard
 * second-order equilibrium (D3Q19-S, Eq. 14 of Bauer & Ruede, arXiv:1803.04937)
 * and the improved equilibrium D3Q19-I (Eq. 22), SRT (Eq. 15) or TRT
 * relaxation (Sec. 3.3), periodic and half-way bounce-back boundaries
 * (Sec. 5.1), a Buick-Greated body force with the velocity shift of Eq. 17,
 * and the reverse-mode adjoint of the step.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Lattice units: dx = dt = 1, c_s^2 = 1/3, omega = 1/tau.
 *  - Every call returns an int status (LBM_OK or an LBM_E* code) and never
 *    throws.  lbm_last_error() gives a message for the last failure on a handle.
 *  - Device memory is owned by the caller.  The library never allocates device
 *    memory: the caller allocates the population grids and a scratch buffer of
 *    the sizes lbm_required_bytes() reports and lends them through lbm_bind().
 *    All device pointers must stay valid until they are re-bound or the handle
 *    is destroyed, and must be 256-byte aligned.
 *  - All GPU work is enqueued on the bound CUDA stream and is asynchronous,
 *    except where a function says it synchronises.
 *  - Macroscopic fields are dense arrays, x fastest:
 *      rho[nz][ny][nx],  u[3][nz][ny][nx]   (u[0] = u_x plane first),
 *    in the element type named by a LBM_DTYPE_* argument.
 *  - Population storage ("PDF grid"): structure of arrays, shifted values
 *      pdf[q][nz][ny][nx] = f_q - w_q
 *    in the storage precision chosen at creation, q in the library's own
 *    D3Q19 order (lbm_velocity_set()).  A grid is 19 * nx * ny * nz elements.
 *  - Not thread-safe per handle; distinct handles are independent.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 1

typedef struct lbm_ctx *lbm_handle;

/* status codes */
#define LBM_OK            0
#define LBM_EINVAL        1  /* bad argument (null pointer, size, key, value) */
#define LBM_ENOMEM        2  /* host allocation of the handle failed */
#define LBM_ECUDA         3  /* a CUDA runtime call or kernel launch failed */
#define LBM_EUNSUPPORTED  4  /* valid request the library does not implement */
#define LBM_ENONFINITE    5  /* lbm_reduce found NaN or Inf in the state */
#define LBM_ESTATE        6  /* call out of order (e.g. lbm_step before lbm_bind) */

/* stencil */
#define LBM_D3Q19 19
#define LBM_D3Q27 27   /* comparison lattice (Sec. 2.3): A/B step, init, moments, copies */

/* equilibrium (Eq. 14 second-order part / Eq. 22) */
#define LBM_EQ_STANDARD 0
#define LBM_EQ_IMPROVED 1

/* collision */
#define LBM_SRT 0
#define LBM_TRT 1
/* MRT (Sec. 3.2-3.3, D3Q19 only): relaxation in the moment space of the
 * monomials xi_x^a xi_y^b xi_z^c (a, b, c in {0,1,2}, without the eight that
 * Eq. 21 drops), against the Maxwellian's moments truncated at second order
 * (LBM_EQ_IMPROVED, which equals Eq. 22 in population space) or against the
 * moments of Eq. 14 (LBM_EQ_STANDARD).  Rates: odd moments omega- (from the
 * magic parameter, as TRT), deviatoric second-order moments omega+ = 1/tau,
 * the trace of the second-order moments LBM_OPT_MRT_OMEGA_BULK, the
 * fourth-order moments LBM_OPT_MRT_OMEGA_4.  Force: (I - S/2) applied in
 * moment space.  With both extra rates equal to 1/tau it is LBM_TRT.  Not
 * every pair of rates is linearly stable (e.g. omega_bulk = 1.9 with
 * omega_4 = 1 at tau = 0.6 is not); the library does not check. */
#define LBM_MRT 2

/* storage precision of the populations (S = shifted storage f_q - w_q);
 * collision arithmetic is FP64 for LBM_F64 and FP32 otherwise. */
#define LBM_F64   0
#define LBM_F32   1
#define LBM_F16S  2
#define LBM_BF16S 3

/* element type of macroscopic field buffers */
#define LBM_DTYPE_F64 0
#define LBM_DTYPE_F32 1

/* propagation pattern */
#define LBM_PATTERN_AB 0   /* two grids, pull stream + collide */
#define LBM_PATTERN_AA 1   /* one grid, in-place AA (even / odd steps) */

/* option keys for lbm_set_option / lbm_get_option */
#define LBM_OPT_TRT_MAGIC  1  /* Lambda = (tau+ - 1/2)(tau- - 1/2); default 3/16 */
#define LBM_OPT_FORCE_X    2  /* body force a_x; default 0 */
#define LBM_OPT_FORCE_Y    3
#define LBM_OPT_FORCE_Z    4
#define LBM_OPT_WALLS_X    5  /* 1: half-way bounce-back walls at both x ends; 0: periodic (default) */
#define LBM_OPT_WALLS_Y    6
#define LBM_OPT_WALLS_Z    7
#define LBM_OPT_RHO0_MODE  8  /* 0: rho0 = 1 (default, Sec. 2.3); 1: rho0 = rho */
#define LBM_OPT_PATTERN    9  /* LBM_PATTERN_AB (default) or LBM_PATTERN_AA */
#define LBM_OPT_TAU       10  /* relaxation time tau (> 1/2) */
#define LBM_OPT_EQUILIBRIUM 11 /* LBM_EQ_STANDARD or LBM_EQ_IMPROVED */
#define LBM_OPT_COLLISION 12  /* LBM_SRT, LBM_TRT or LBM_MRT (D3Q19) */
#define LBM_OPT_BLOCK_X   13  /* step kernel threads per block along x (tuning) */
#define LBM_OPT_BLOCK_Y   14  /* ... along y; bx * by <= 256 and a multiple of 32 */
#define LBM_OPT_CELLS_X   15  /* cells per thread along x in the step kernel: 1; 2 (paired
                                 accesses; nx even, bx a multiple of 32); or 4 (16-bit storage,
                                 A/B and AA, nx a multiple of 4, 128-thread blocks shaped from
                                 nx; otherwise treated as 2).  Default 4 for 16-bit storage, 1
                                 otherwise.  LBM_MRT runs one cell per thread except with 4. */
#define LBM_OPT_MRT_OMEGA_BULK 16 /* LBM_MRT: rate of the trace of the second-order moments
                                     (bulk viscosity (2/9)(1/omega - 1/2)); 0 < v < 2, default 1 */
#define LBM_OPT_MRT_OMEGA_4    17 /* LBM_MRT: rate of the fourth-order moments; 0 < v < 2,
                                     default 1 */
#define LBM_OPT_GRAPHS    18  /* 1 (default): lbm_step replays captured CUDA graphs of 16 steps
                                 (built on first use from the current grid or parity, dropped
                                 by lbm_set_option and lbm_bind; not used while the bound stream
                                 is being captured by the caller); 0: one launch per step.
                                 Same results either way. */
#define LBM_OPT_ADJ_DEFER_SUM 19  /* 0 (default): each lbm_adjoint_step adds its dL/domega
                                 terms to its grad_omega before the call's work ends; 1:
                                 the terms of a step are summed by the next lbm_adjoint_step
                                 (in the first block of its kernel) or by lbm_adjoint_flush,
                                 which takes a one-block kernel off each step's critical path.
                                 Bitwise the same sums either way.  Changing the option,
                                 lbm_bind with another scratch buffer or stream, lbm_reduce,
                                 lbm_enstrophy and lbm_adjoint_seed flush first; lbm_destroy
                                 drops a pending sum. */

/* lbm_reduce output slots */
#define LBM_RED_MASS      0   /* sum_x rho */
#define LBM_RED_ENERGY    1   /* 1/2 sum_x |u|^2 */
#define LBM_RED_JX        2   /* sum_x sum_q c_qx f_q */
#define LBM_RED_JY        3
#define LBM_RED_JZ        4
#define LBM_RED_UMAX      5   /* max_x |u| */
#define LBM_RED_NONFINITE 6   /* number of cells with a non-finite population */
#define LBM_RED_COUNT     8

/* Library ABI version (LBM_ABI_VERSION of the build). Host only. */
int lbm_abi_version(void);

/* Static string for a status code. Host only. */
const char *lbm_status_string(int status);

/* The library's D3Q19 order (Sec. 2.3 fixes only the three groups):
 * c[3*q + i] (ints), w[q], opp[q] (index of -c_q).  Any pointer may be NULL.
 * Host only. */
int lbm_velocity_set(int *c, double *w, int *opp);

/* The same for a stencil (LBM_D3Q19 or LBM_D3Q27; Q = the stencil value):
 * c[3*q + i], w[q], opp[q] for q < Q.  Host only. */
int lbm_velocity_set_of(int stencil, int *c, double *w, int *opp);

/*
 * Creates a handle for an nx * ny * nz lattice (Sec. 2.3 lattice, Eq. 15 update).
 *   stencil      LBM_D3Q19, or LBM_D3Q27 (standard equilibrium, Eq. 14, for either
 *                equilibrium choice: the construction of Sec. 3.1 gives Eq. 14
 *                on D3Q27; A/B pattern only; lbm_reduce, lbm_reduce_noalloc and
 *                the adjoint return LBM_EUNSUPPORTED)
 *   equilibrium  LBM_EQ_STANDARD (Eq. 14, second order) | LBM_EQ_IMPROVED (Eq. 22)
 *   collision    LBM_SRT (Eq. 15) | LBM_TRT (magic parameter LBM_OPT_TRT_MAGIC) |
 *                LBM_MRT (D3Q19 only; LBM_EUNSUPPORTED with LBM_D3Q27)
 *   tau          relaxation time, > 1/2
 *   precision    LBM_F64 | LBM_F32 | LBM_F16S | LBM_BF16S
 * Sizes: each >= 1, nx * ny * nz < 2^31.  Host only (no CUDA call).
 * On success *out receives the handle; on failure *out is set to NULL.
 */
int lbm_create(int nx, int ny, int nz, int stencil, int equilibrium, int collision,
               double tau, int precision, lbm_handle *out);

/* Frees the handle (host metadata only; borrowed device memory is untouched). */
int lbm_destroy(lbm_handle h);

/* Sets / reads an option (LBM_OPT_*).  Host only; takes effect at the next launch. */
int lbm_set_option(lbm_handle h, int key, double value);
int lbm_get_option(lbm_handle h, int key, double *value);

/*
 * Device memory the caller must provide:
 *   *pdf_bytes_per_grid  bytes of one PDF grid (19 * cells * element size)
 *   *n_grids             2 for LBM_PATTERN_AB, 1 for LBM_PATTERN_AA
 *   *scratch_bytes       bytes of the scratch buffer used by lbm_reduce,
 *                        lbm_enstrophy and lbm_adjoint_step (FP64 block partials;
 *                        two buffers of adjoint partials for deferred sums)
 * Any pointer may be NULL.  Host only.
 */
int lbm_required_bytes(lbm_handle h, size_t *pdf_bytes_per_grid, int *n_grids,
                       size_t *scratch_bytes);

/*
 * Lends device memory and a stream (a cudaStream_t, NULL = legacy default).
 *   pdf_a    grid that holds (or will hold) the current state
 *   pdf_b    second grid for LBM_PATTERN_AB; ignored (may be NULL) for AA
 *   scratch  scratch buffer of at least scratch_bytes, or NULL (then
 *            lbm_reduce and lbm_adjoint_step return LBM_ESTATE)
 * Re-binding is allowed at any time between calls and makes pdf_a the current
 * state; the step counter and, for AA, the parity are kept, so a state copied
 * out of the current grid can be restored by binding a grid that holds it.
 */
int lbm_bind(lbm_handle h, void *pdf_a, void *pdf_b, void *scratch, void *stream);

/*
 * Sets the state to f_q = f_q^eq(rho, u) for the configured equilibrium
 * (Eq. 14 or Eq. 22; no non-equilibrium part) and resets the step counter.
 * rho, u: buffers of element type dtype; rho may be NULL (rho = 1).  Either
 * may be device memory or pinned (page-locked) host memory: the kernel then
 * reads the host buffer directly through its mapped device address, with no
 * staging copy, and the buffer must stay valid until the stream has passed
 * the call.  Pageable host memory returns LBM_EINVAL.
 */
int lbm_init(lbm_handle h, const void *rho, const void *u, int dtype);

/*
 * Enqueues n >= 0 time steps of Eq. 15 (stream + collide) on the bound stream.
 * A caller may capture these launches into its own CUDA graph by capturing
 * the bound stream (the library then launches plain kernels, see
 * LBM_OPT_GRAPHS); a replayed capture advances the state but not the step
 * counter of lbm_steps_done, and an even n keeps the grid / parity bookkeeping
 * of the handle consistent across replays.
 */
int lbm_step(lbm_handle h, int n);

/*
 * Writes rho (Eq. 16) and u (Eq. 17: rho0 u = sum_q c_q f_q + a/2) of the
 * current state into buffers of element type dtype.  Either output may be
 * NULL.  As for lbm_init, an output may be device memory or pinned host memory
 * (written directly by the kernel; complete once the bound stream has passed
 * the call); pageable host memory returns LBM_EINVAL.
 */
int lbm_moments(lbm_handle h, void *rho, void *u, int dtype);

/*
 * FP64 reductions of the current state into host out[LBM_RED_COUNT] (slots
 * LBM_RED_*), deterministic for a given lattice size.  Needs a bound scratch
 * buffer.  Synchronises the bound stream.  Returns LBM_ENONFINITE (with out
 * filled) if any population is NaN or Inf.
 */
int lbm_reduce(lbm_handle h, double *out);

/*
 * Enstrophy of the current state into host *out: 1/2 <|curl u|^2>, the mean
 * over all cells, with u from Eq. 17 and second-order central differences
 * (u(x + e_a) - u(x - e_a)) / 2.  Periodic axes wrap; across a half-way
 * bounce-back wall the ghost velocity is -u of the own cell.  FP64
 * accumulation, deterministic for a given lattice size.  Needs a bound scratch
 * buffer; synchronises the bound stream.  D3Q19 only.  Off the per-step path:
 * each cell reads its six axis neighbours' populations.  Returns
 * LBM_ENONFINITE if the result is not finite.
 */
int lbm_enstrophy(lbm_handle h, double *out);

/*
 * lbm_reduce without a scratch buffer: the same FP64 reductions of the
 * current state into host out[LBM_RED_COUNT], for callers that cannot
 * allocate device memory (for example a host application that hands the
 * library a fixed memory budget, or code running where cudaMalloc is not
 * allowed).  The paper has no counterpart; this is an interface convenience.
 *
 * Its scratch is a static device array of the library (64 KiB: FP64 partial
 * sums of up to 1024 reduction blocks, plus the results), held on every GPU
 * that loads the library until the process exits.  The reduction grid does
 * not depend on the lattice size, so every lattice lbm_create accepts fits;
 * should the reduction ever need more rows than the array holds, the call
 * returns LBM_EUNSUPPORTED with a message.  It calls no allocating routine.
 * Every call looks the array's device address up (cudaGetSymbolAddress) with
 * the calling thread's current device, which must be the device of the bound
 * stream (LBM_EINVAL otherwise); so the address stays right after the caller
 * has reset the device (cudaDeviceReset) and re-bound fresh buffers.  The
 * first lookup on a device may load the library's device code; make the
 * first call on a device before any stream capture.  All calls share the array and every call
 * rewrites the parts it reads, so no clearing is needed, but calls that
 * overlap on the GPU (other streams, other handles) race on it.  Needs
 * lbm_bind (grids and stream; the scratch pointer may be NULL).
 * Synchronises the bound stream.  Returns LBM_ENONFINITE like lbm_reduce.
 */
int lbm_reduce_noalloc(lbm_handle h, double *out);

/* Step counter (number of lbm_step time steps since lbm_init / lbm_set_pdfs). */
int lbm_steps_done(lbm_handle h, long long *t);

/*
 * Copies the current state, in canonical order (f_q(x, t) - w_q at
 * dst[q][z][y][x], storage precision), to the device buffer dst (one grid),
 * whatever the propagation pattern.  lbm_set_pdfs is the inverse and makes
 * the state exactly the given populations (bitwise round trip).
 */
int lbm_get_pdfs(lbm_handle h, void *dst);
int lbm_set_pdfs(lbm_handle h, const void *src);

/*
 * Adjoint (reverse-mode derivative) of the time step, rho0 = 1 only
 * (LBM_EUNSUPPORTED otherwise).  Not in the paper: the derivative of Eq. 15
 * (or its TRT form) with respect to the populations and to omega.
 *
 * lambda buffers hold dL/df_q(x, t) in natural order lambda[q][z][y][x], as
 * double for LBM_F64 and float for the other precisions.
 *
 * lbm_adjoint_seed: lambda(T) from dL/du(T) (grad_u, [3][nz][ny][nx]) and
 *   optionally dL/drho(T) (grad_rho, may be NULL), dtype LBM_DTYPE_*:
 *   lambda_q = c_q . grad_u + grad_rho.
 *
 * lbm_adjoint_step: lambda_t = (d state(t+1) / d state(t))^T lambda_next for
 *   the step that took state_t to state t+1, and adds the step's
 *   contributions to dL/d omega+ and dL/d omega- to the two device doubles
 *   grad_omega[0..1] (FP64, deterministic order).  state_t is a PDF grid in
 *   the A/B layout exactly as the forward pass left it in the current grid
 *   (lbm_bind + lbm_step with LBM_PATTERN_AB), i.e. a checkpoint copy of it.
 *   lambda_next and lambda_t must not overlap.  Needs a bound scratch buffer.
 *   With LBM_OPT_ADJ_DEFER_SUM = 1 the step's contributions reach grad_omega
 *   only when the next lbm_adjoint_step's kernel or lbm_adjoint_flush has run
 *   on the stream (the block partials wait in the scratch buffer).
 *
 * lbm_adjoint_flush: adds the contributions of a deferred step (if any) to its
 *   grad_omega; enqueued on the bound stream.
 *
 * lbm_adjoint_init_velocity: dL/du0 from lambda(0) through f(0) =
 *   f^eq(rho, u0) (lbm_init).  rho may be NULL (rho = 1); grad_u0 has dtype.
 *
 * lbm_adjoint_tau_gradient: dL/dtau = dL/domega+ domega+/dtau +
 *   dL/domega- domega-/dtau for the handle's tau, collision and magic
 *   parameter, from host copies of grad_omega.  Host only.
 *
 * The adjoint covers LBM_SRT and LBM_TRT; with LBM_MRT every adjoint entry
 * point returns LBM_EUNSUPPORTED.
 */
int lbm_adjoint_seed(lbm_handle h, const void *grad_rho, const void *grad_u, int dtype,
                     void *lambda);
int lbm_adjoint_step(lbm_handle h, const void *state_t, const void *lambda_next,
                     void *lambda_t, double *grad_omega);
int lbm_adjoint_flush(lbm_handle h);
int lbm_adjoint_init_velocity(lbm_handle h, const void *rho, const void *u0, int dtype,
                              const void *lambda0, void *grad_u0);
int lbm_adjoint_tau_gradient(lbm_handle h, const double *grad_omega, double *dL_dtau);

/* Message for the last failing call on h (empty string if none). */
const char *lbm_last_error(lbm_handle h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
