// Kernels around the time step: initialisation f = feq(rho, u), macroscopic
// moments (Eq. 16, Eq. 17), canonical copies of the state, and the FP64
// global reductions (mass, kinetic energy, momentum, max |u|, non-finite count).

#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace lbm {

static dim3 cell_block() { return dim3(128, 2, 1); }
static dim3 cell_grid(const Geo &g)
{
    return dim3((g.nx + 127) / 128, (g.ny + 1) / 2, g.nz);
}

#define LBM_CELL_PROLOGUE                                          \
    const int x = blockIdx.x * blockDim.x + threadIdx.x;           \
    const int y = blockIdx.y * blockDim.y + threadIdx.y;           \
    const int z = blockIdx.z;                                      \
    if (x >= g.nx || y >= g.ny) return;                            \
    Cell c(x, y, z, g);                                            \
    const long long cell = c.self();

// ---------------------------------------------------------------- init

template <typename T, typename In, int D>
__global__ void k_init(T *grid, const In *rho, const In *u, Geo g, Coll<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    LBM_CELL_PROLOGUE
    R r = rho ? R(rho[cell]) : R(1);
    R uv[3] = {R(u[cell]), R(u[g.ncell + cell]), R(u[2 * g.ncell + cell])};
    R f[Q];
    equilibrium_all(r, uv, p, f);
    scatter<D>(grid, c, g.ncell, f);
}

template <typename T, typename In>
static cudaError_t init_t(int layout, void *grid, const void *rho, const void *u, const Geo &g, const CollBoth &cb,
                          cudaStream_t s)
{
    using R = typename Storage<T>::R;
    Coll<R> p = to_coll<R>(cb);
    if (layout == AB)
        k_init<T, In, D_AB_CANON><<<cell_grid(g), cell_block(), 0, s>>>((T *)grid, (const In *)rho, (const In *)u, g, p);
    else
        k_init<T, In, D_AB_NEXT><<<cell_grid(g), cell_block(), 0, s>>>((T *)grid, (const In *)rho, (const In *)u,
                                                                       g, p);  // natural order = AA even layout
    return cudaGetLastError();
}

// ---------------------------------------------------------------- moments

template <typename T, typename Out, int L>
__global__ void k_moments(const T *__restrict__ grid, Out *rho, Out *u, Geo g, Coll<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    LBM_CELL_PROLOGUE
    R f[Q];
    gather<L>(grid, c, g.ncell, f);
    R drho, rho0, uv[3];
    macro(f, p, drho, rho0, uv);
    if (rho) rho[cell] = Out(R(1) + drho);
    if (u) {
        u[cell] = Out(uv[0]);
        u[g.ncell + cell] = Out(uv[1]);
        u[2 * g.ncell + cell] = Out(uv[2]);
    }
}

// ---------------------------------------------------------------- canonical copies

template <typename T, int L>
__global__ void k_get(const T *__restrict__ grid, T *__restrict__ dst, Geo g)
{
    LBM_CELL_PROLOGUE
    const int self = (int)cell;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        long long off;
        if (L == AA_EVEN) {
            off = (long long)q * g.ncell + self;
        } else {
            bool wall;
            int src = c.template along<-1>(q, wall);
            if (L == AB)
                off = wall ? (long long)OPP(q) * g.ncell + self : (long long)q * g.ncell + src;
            else
                off = wall ? (long long)q * g.ncell + self : (long long)OPP(q) * g.ncell + src;
        }
        dst[(long long)q * g.ncell + self] = grid[off];
    }
}

// CANON_AB = 1: write so that the AB gather returns src; 0: natural order
// (the AA even layout).
template <typename T, int CANON_AB>
__global__ void k_set(T *grid, const T *__restrict__ src, Geo g)
{
    LBM_CELL_PROLOGUE
    const int self = (int)cell;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        long long off;
        if (!CANON_AB) {
            off = (long long)q * g.ncell + self;
        } else {
            bool wall;
            int dst = c.template along<-1>(q, wall);
            off = wall ? (long long)OPP(q) * g.ncell + self : (long long)q * g.ncell + dst;
        }
        grid[off] = src[(long long)q * g.ncell + self];
    }
}

// ---------------------------------------------------------------- reductions

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 152 * 4;
int reduce_blocks() { return RED_BLOCKS; }

template <typename T, int L>
__global__ void __launch_bounds__(RED_THREADS) k_reduce(const T *__restrict__ grid, double *partial, Geo g,
                                                        Coll<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    __shared__ double sh[32];
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const long long nxy = (long long)g.nx * g.ny;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell;
         cell += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(cell / nxy);
        const int rem = (int)(cell - z * nxy);
        const int y = rem / g.nx;
        const int x = rem - y * g.nx;
        Cell c(x, y, z, g);
        R f[Q];
        gather<L>(grid, c, g.ncell, f);
        bool bad = false;
#pragma unroll
        for (int q = 0; q < Q; ++q) bad |= !isfinite(f[q]);
        R drho, rho0, uv[3];
        macro(f, p, drho, rho0, uv);
        double u0 = uv[0], u1 = uv[1], u2 = uv[2];
        double r0 = rho0;
        double uu = u0 * u0 + u1 * u1 + u2 * u2;
        acc[0] += (double)drho;
        acc[1] += 0.5 * uu;
        acc[2] += r0 * u0 - (double)p.half_a[0];
        acc[3] += r0 * u1 - (double)p.half_a[1];
        acc[4] += r0 * u2 - (double)p.half_a[2];
        acc[5] = fmax(acc[5], sqrt(uu));
        acc[6] += bad ? 1.0 : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        double v = (k == 5) ? block_max(acc[k], sh) : block_sum(acc[k], sh);
        if (threadIdx.x == 0) partial[blockIdx.x * 8 + k] = v;
    }
}

__global__ void __launch_bounds__(RED_THREADS) k_reduce_final(const double *partial, int nblocks, double *result,
                                                              double ncell)
{
    __shared__ double sh[32];
    for (int k = 0; k < 7; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
            v = (k == 5) ? fmax(v, partial[b * 8 + k]) : v + partial[b * 8 + k];
        v = (k == 5) ? block_max(v, sh) : block_sum(v, sh);
        if (threadIdx.x == 0) result[k] = (k == 0) ? ncell + v : v;
    }
    if (threadIdx.x == 0) result[7] = 0.0;
}

// Enstrophy 1/2 <|curl u|^2> of the state, with second-order central
// differences of u (Eq. 17) between the axis neighbours.  Periodic axes wrap;
// across a half-way bounce-back wall the ghost velocity is -u of the own cell
// (the wall at rest halfway between them).  Each cell gathers its six
// neighbours' populations (off the per-step path; the neighbours' rows are
// shared through L1/L2).  Deterministic: fixed grid, fixed per-thread order,
// fixed trees.
template <typename T, int L>
__device__ __forceinline__ void velocity_at(const T *__restrict__ grid, int x, int y, int z, const Geo &g,
                                            const Coll<typename Storage<T>::R> &p, double u[3])
{
    using R = typename Storage<T>::R;
    const Cell c(x, y, z, g);
    R f[Q];
    gather<L>(grid, c, g.ncell, f);
    R drho, rho0, uv[3];
    macro(f, p, drho, rho0, uv);
    u[0] = uv[0];
    u[1] = uv[1];
    u[2] = uv[2];
}

template <typename T, int L>
__global__ void __launch_bounds__(RED_THREADS) k_enstrophy(const T *__restrict__ grid, double *partial, Geo g,
                                                           Coll<typename Storage<T>::R> p)
{
    __shared__ double sh[32];
    double acc = 0.0;
    const long long nxy = (long long)g.nx * g.ny;
    const int n[3] = {g.nx, g.ny, g.nz};
    const bool wall[3] = {g.wall_x != 0, g.wall_y != 0, g.wall_z != 0};
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell;
         cell += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(cell / nxy);
        const int rem = (int)(cell - z * nxy);
        const int y = rem / g.nx;
        const int x = rem - y * g.nx;
        const int pos[3] = {x, y, z};
        double own[3];
        velocity_at<T, L>(grid, x, y, z, g, p, own);
        // D[a][i] = (u_i(x + e_a) - u_i(x - e_a)) / 2
        double D[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double up[3], um[3];
            int qp[3] = {x, y, z}, qm[3] = {x, y, z};
            const bool wp = wall[a] && pos[a] == n[a] - 1, wm = wall[a] && pos[a] == 0;
            qp[a] = pos[a] == n[a] - 1 ? 0 : pos[a] + 1;
            qm[a] = pos[a] == 0 ? n[a] - 1 : pos[a] - 1;
            if (wp) { up[0] = -own[0]; up[1] = -own[1]; up[2] = -own[2]; }
            else velocity_at<T, L>(grid, qp[0], qp[1], qp[2], g, p, up);
            if (wm) { um[0] = -own[0]; um[1] = -own[1]; um[2] = -own[2]; }
            else velocity_at<T, L>(grid, qm[0], qm[1], qm[2], g, p, um);
#pragma unroll
            for (int i = 0; i < 3; ++i) D[a][i] = 0.5 * (up[i] - um[i]);
        }
        const double wx = D[1][2] - D[2][1];
        const double wy = D[2][0] - D[0][2];
        const double wz = D[0][1] - D[1][0];
        acc += wx * wx + wy * wy + wz * wz;
    }
    const double v = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x * 8] = v;
}

__global__ void __launch_bounds__(RED_THREADS) k_enstrophy_final(const double *partial, int nblocks,
                                                                 double *result, double ncell)
{
    __shared__ double sh[32];
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[b * 8];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) result[0] = 0.5 * v / ncell;
}

// ---------------------------------------------------------------- dispatch

template <typename F>
static cudaError_t by_prec(int prec, F &&f)
{
    switch (prec) {
    case P_F64: return f(double());
    case P_F32: return f(float());
    case P_F16: return f(__half());
    case P_BF16: return f(__nv_bfloat16());
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_init(int prec, int layout, void *grid, const void *rho, const void *u, int dtype, const Geo &g,
                        const CollBoth &c, cudaStream_t s)
{
    return by_prec(prec, [&](auto t) {
        using T = decltype(t);
        return dtype == 0 ? init_t<T, double>(layout, grid, rho, u, g, c, s)
                          : init_t<T, float>(layout, grid, rho, u, g, c, s);
    });
}

cudaError_t launch_moments(int prec, int layout, const void *grid, void *rho, void *u, int dtype, const Geo &g,
                           const CollBoth &cb, cudaStream_t s)
{
    return by_prec(prec, [&](auto t) {
        using T = decltype(t);
        using R = typename Storage<T>::R;
        Coll<R> p = to_coll<R>(cb);
        const T *gr = (const T *)grid;
        if (dtype == 0) {
            double *r = (double *)rho, *uu = (double *)u;
            if (layout == AB) k_moments<T, double, AB><<<cell_grid(g), cell_block(), 0, s>>>(gr, r, uu, g, p);
            else if (layout == AA_EVEN) k_moments<T, double, AA_EVEN><<<cell_grid(g), cell_block(), 0, s>>>(gr, r, uu, g, p);
            else k_moments<T, double, AA_ODD><<<cell_grid(g), cell_block(), 0, s>>>(gr, r, uu, g, p);
        } else {
            float *r = (float *)rho, *uu = (float *)u;
            if (layout == AB) k_moments<T, float, AB><<<cell_grid(g), cell_block(), 0, s>>>(gr, r, uu, g, p);
            else if (layout == AA_EVEN) k_moments<T, float, AA_EVEN><<<cell_grid(g), cell_block(), 0, s>>>(gr, r, uu, g, p);
            else k_moments<T, float, AA_ODD><<<cell_grid(g), cell_block(), 0, s>>>(gr, r, uu, g, p);
        }
        return cudaGetLastError();
    });
}

cudaError_t launch_get_pdfs(int prec, int layout, const void *grid, void *dst, const Geo &g, cudaStream_t s)
{
    return by_prec(prec, [&](auto t) {
        using T = decltype(t);
        const T *gr = (const T *)grid;
        T *d = (T *)dst;
        if (layout == AB) k_get<T, AB><<<cell_grid(g), cell_block(), 0, s>>>(gr, d, g);
        else if (layout == AA_EVEN) k_get<T, AA_EVEN><<<cell_grid(g), cell_block(), 0, s>>>(gr, d, g);
        else k_get<T, AA_ODD><<<cell_grid(g), cell_block(), 0, s>>>(gr, d, g);
        return cudaGetLastError();
    });
}

cudaError_t launch_set_pdfs(int prec, int layout, void *grid, const void *src, const Geo &g, cudaStream_t s)
{
    return by_prec(prec, [&](auto t) {
        using T = decltype(t);
        T *gr = (T *)grid;
        const T *sr = (const T *)src;
        if (layout == AB) k_set<T, 1><<<cell_grid(g), cell_block(), 0, s>>>(gr, sr, g);
        else k_set<T, 0><<<cell_grid(g), cell_block(), 0, s>>>(gr, sr, g);
        return cudaGetLastError();
    });
}

cudaError_t launch_reduce(int prec, int layout, const void *grid, double *scratch, double *result, const Geo &g,
                          const CollBoth &cb, cudaStream_t s)
{
    cudaError_t e = by_prec(prec, [&](auto t) {
        using T = decltype(t);
        using R = typename Storage<T>::R;
        Coll<R> p = to_coll<R>(cb);
        const T *gr = (const T *)grid;
        if (layout == AB) k_reduce<T, AB><<<RED_BLOCKS, RED_THREADS, 0, s>>>(gr, scratch, g, p);
        else if (layout == AA_EVEN) k_reduce<T, AA_EVEN><<<RED_BLOCKS, RED_THREADS, 0, s>>>(gr, scratch, g, p);
        else k_reduce<T, AA_ODD><<<RED_BLOCKS, RED_THREADS, 0, s>>>(gr, scratch, g, p);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, RED_THREADS, 0, s>>>(scratch, RED_BLOCKS, result, (double)g.ncell);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- reduction without caller scratch
//
// lbm_reduce_noalloc serves callers that cannot allocate device memory (for
// example code running inside an allocator-less host, or a caller whose
// memory budget is fixed up front): its FP64 block partials and results live
// in this file-scope array instead of the scratch buffer lent to lbm_bind.
// Every GPU that loads the library holds the array until the process exits.
// In host code `g_reduce_scratch` only names a host-side stand-in; the device
// address is looked up with cudaGetSymbolAddress on every call, with the
// calling thread's current device, which must be the device of the bound
// stream (checked).  Looking it up each time keeps it right after the
// primary context has been destroyed and created again (cudaDeviceReset); the
// first lookup on a device may load the library's module, so the first call
// on a device should come before any stream capture.  All calls share the
// array and each call overwrites all of it that it reads (every block writes
// its partial row, the final kernel writes the results), so nothing needs
// clearing between calls; calls that overlap on the GPU (several streams or
// handles at once) race on it.
constexpr int NOALLOC_MAX_BLOCKS = 1024;                 // partial rows the array holds
constexpr int NOALLOC_DOUBLES = NOALLOC_MAX_BLOCKS * 8 + 8;  // 64 KiB + results
static __device__ __align__(256) double g_reduce_scratch[NOALLOC_DOUBLES];

int reduce_noalloc_capacity_doubles() { return NOALLOC_DOUBLES; }

cudaError_t launch_enstrophy(int prec, int layout, const void *grid, double *scratch, double *result, const Geo &g,
                             const CollBoth &c, cudaStream_t s)
{
    cudaError_t e = by_prec(prec, [&](auto tag) {
        using T = decltype(tag);
        using R = typename Storage<T>::R;
        const Coll<R> p = to_coll<R>(c);
        const T *gr = static_cast<const T *>(grid);
        if (layout == AB) k_enstrophy<T, AB><<<RED_BLOCKS, RED_THREADS, 0, s>>>(gr, scratch, g, p);
        else if (layout == AA_EVEN) k_enstrophy<T, AA_EVEN><<<RED_BLOCKS, RED_THREADS, 0, s>>>(gr, scratch, g, p);
        else k_enstrophy<T, AA_ODD><<<RED_BLOCKS, RED_THREADS, 0, s>>>(gr, scratch, g, p);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    k_enstrophy_final<<<1, RED_THREADS, 0, s>>>(scratch, RED_BLOCKS, result, (double)g.ncell);
    return cudaGetLastError();
}

cudaError_t launch_reduce_noalloc(int prec, int layout, const void *grid, const Geo &g, const CollBoth &c,
                                  cudaStream_t s, double **result)
{
    if ((long long)RED_BLOCKS * 8 + 8 > NOALLOC_DOUBLES) return cudaErrorInvalidValue;
    int dev = -1, sdev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaStreamGetDevice(s, &sdev);
    if (e != cudaSuccess) return e;
    if (sdev != dev) return cudaErrorInvalidDevice;
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_reduce_scratch);
    if (e != cudaSuccess) return e;
    double *base = static_cast<double *>(p);
    *result = base + (size_t)RED_BLOCKS * 8;
    return launch_reduce(prec, layout, grid, base, *result, g, c, s);
}

}  // namespace lbm
