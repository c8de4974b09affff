// Host-side launch interface between the C ABI (lbm_api.cu) and the kernels.
// Every launcher enqueues on `stream` and returns the cudaError_t of the launch.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct Geo;
template <typename R> struct Coll;

enum Prec { P_F64 = 0, P_F32 = 1, P_F16 = 2, P_BF16 = 3 };

// Layout of the current state (see lbm_device.cuh): 0 AB, 1 AA even, 2 AA odd.
struct LaunchShape {
    int bx, by;   // thread block (bx * by threads, bx along x)
    int cells_x;  // cells per thread along x: 1, or 2 (used when nx is even)
};

// Collision constants for both arithmetic types; the launcher picks one.
struct CollBoth {
    double omega_p, omega_m, kappa;
    double omega_bulk, omega_4;  // MRT rates (equal to omega_p otherwise)
    int mrt;                     // 1: MRT collision (one cell per thread)
    double half_a[3];
    double force[9];
    int rho0_is_rho;
};

// One time step.  kind: 0 AB (src -> dst), 1 AA even (in place), 2 AA odd (in place).
cudaError_t launch_step(int prec, int kind, const void *src, void *dst, const Geo &g, const CollBoth &c,
                        LaunchShape s, cudaStream_t stream);

// f = feq(rho, u) written into `grid` for layout (0: AB, 1: AA even).
cudaError_t launch_init(int prec, int layout, void *grid, const void *rho, const void *u, int dtype,
                        const Geo &g, const CollBoth &c, cudaStream_t stream);

// rho, u (Eq. 16, 17) of the state in `grid` with `layout` (0 AB, 1 AA even, 2 AA odd).
cudaError_t launch_moments(int prec, int layout, const void *grid, void *rho, void *u, int dtype,
                           const Geo &g, const CollBoth &c, cudaStream_t stream);

// Canonical copy out of / into a state grid.
cudaError_t launch_get_pdfs(int prec, int layout, const void *grid, void *dst, const Geo &g,
                            cudaStream_t stream);
cudaError_t launch_set_pdfs(int prec, int layout, void *grid, const void *src, const Geo &g,
                            cudaStream_t stream);

// FP64 reductions into scratch; the LBM_RED_COUNT results land at scratch_result (device).
int reduce_blocks();
cudaError_t launch_reduce(int prec, int layout, const void *grid, double *scratch, double *scratch_result,
                          const Geo &g, const CollBoth &c, cudaStream_t stream);

// Enstrophy 1/2 <|curl u|^2> (central differences) of the state into result[0].
cudaError_t launch_enstrophy(int prec, int layout, const void *grid, double *scratch, double *result,
                             const Geo &g, const CollBoth &c, cudaStream_t stream);

// The same reduction with its scratch in a static device array (lbm_reduce_noalloc);
// *result receives the device address of the LBM_RED_COUNT results.
int reduce_noalloc_capacity_doubles();
cudaError_t launch_reduce_noalloc(int prec, int layout, const void *grid, const Geo &g, const CollBoth &c,
                                  cudaStream_t s, double **result);

// D3Q27 (A/B pattern only): step, init, moments, canonical copies, velocity set.
cudaError_t launch_step27(int prec, const void *src, void *dst, const Geo &g, const CollBoth &c, LaunchShape s,
                          cudaStream_t stream);
cudaError_t launch_init27(int prec, void *grid, const void *rho, const void *u, int dtype, const Geo &g,
                          const CollBoth &c, cudaStream_t stream);
cudaError_t launch_moments27(int prec, const void *grid, void *rho, void *u, int dtype, const Geo &g,
                             const CollBoth &c, cudaStream_t stream);
cudaError_t launch_get27(int prec, const void *grid, void *dst, const Geo &g, cudaStream_t stream);
cudaError_t launch_set27(int prec, void *grid, const void *src, const Geo &g, cudaStream_t stream);
int velocity_set27(int *c, double *w, int *opp);

// Adjoint kernels (see lbm.h).
int adjoint_blocks(const Geo &g);
cudaError_t launch_adjoint_seed(int prec, const void *grad_rho, const void *grad_u, int dtype, void *lambda,
                                const Geo &g, cudaStream_t stream);
// partial: this step's block partials (adjoint_blocks(g) x 2 doubles); prev_partial / prev_grad (may be NULL):
// a deferred step's partials, summed into prev_grad by this step's first block; defer: leave this step's
// partials for the next step or launch_adjoint_flush instead of summing them into grad_omega at once.
cudaError_t launch_adjoint_step(int prec, const void *state, const void *lam_next, void *lam, double *grad_omega,
                                double *partial, const double *prev_partial, double *prev_grad, bool defer,
                                const Geo &g, const CollBoth &c, cudaStream_t stream);
cudaError_t launch_adjoint_flush(int prec, const double *partial, double *grad_omega, const Geo &g,
                                 cudaStream_t stream);
cudaError_t launch_adjoint_init_velocity(int prec, const void *rho, const void *u0, int dtype, const void *lam0,
                                         void *grad_u0, const Geo &g, const CollBoth &c, cudaStream_t stream);

}  // namespace lbm
