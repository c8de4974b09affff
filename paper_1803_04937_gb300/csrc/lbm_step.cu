// Fused stream + collide time step (Eq. 15; D3Q19-S / D3Q19-I equilibria;
// SRT / TRT; periodic or half-way bounce-back; Buick-Greated force).
//
// Each thread gathers the populations that stream into its cell(s), collides
// them in registers (FP32, or FP64 for FP64 storage) and stores the
// post-collision values.  Structure-of-arrays storage gives coalesced accesses
// along x for every population.  Algorithmic traffic: 19 loads + 19 stores
// per cell.
//
// Two thread mappings:
//  - one cell per thread (any nx): scalar loads; the +-x populations are read
//    one element off alignment, which L1/L2 absorb without extra DRAM traffic.
//  - two neighbouring cells per thread (nx even): every population is read
//    and written as an aligned pair (half2 / bfloat162 / float2 / double2);
//    a +-x shifted pair is assembled from the own pair and one element of the
//    neighbouring lane's pair (warp shuffle), with one scalar load at the
//    warp's edge.  Halves the load/store instructions and the per-cell index
//    arithmetic, which the 16-bit formats need to reach the HBM roofline.
#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace lbm {

// A/B pull step, one cell per thread: gather from src (layout AB), write dst.
template <typename T, bool RHO0>
__global__ void __launch_bounds__(256) k_step_ab(const T *__restrict__ src, T *__restrict__ dst, Geo g,
                                                 Relax<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    Cell c(x, y, z, g);
    R f[Q];
    gather<AB>(src, c, g.ncell, f);
    collide_lean<R, RHO0>(f, p);
    scatter<D_AB_NEXT>(dst, c, g.ncell, f);
}

// ---------------------------------------------------------------- pairs

template <typename T> struct Pair;
template <> struct Pair<float> {
    static __device__ __forceinline__ void load(const float *p, float &a, float &b)
    {
        float2 v = *reinterpret_cast<const float2 *>(p);
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void store(float *p, float a, float b)
    {
        *reinterpret_cast<float2 *>(p) = make_float2(a, b);
    }
};
template <> struct Pair<double> {
    static __device__ __forceinline__ void load(const double *p, double &a, double &b)
    {
        double2 v = *reinterpret_cast<const double2 *>(p);
        a = v.x;
        b = v.y;
    }
    static __device__ __forceinline__ void store(double *p, double a, double b)
    {
        *reinterpret_cast<double2 *>(p) = make_double2(a, b);
    }
};
template <> struct Pair<__half> {
    static __device__ __forceinline__ void load(const __half *p, float &a, float &b)
    {
        __half2 v = *reinterpret_cast<const __half2 *>(p);
        a = __low2float(v);
        b = __high2float(v);
    }
    static __device__ __forceinline__ void store(__half *p, float a, float b)
    {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
    }
};
template <> struct Pair<__nv_bfloat16> {
    static __device__ __forceinline__ void load(const __nv_bfloat16 *p, float &a, float &b)
    {
        __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(p);
        a = __low2float(v);
        b = __high2float(v);
    }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, float a, float b)
    {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
    }
};

// Pair-wise gather for two cells (x0, x0 + 1), x0 even, nx even, of the
// populations that stream into them.  SWAP = false: A/B layout (plane q at
// x - c_q, through a wall plane qbar of the own cell); SWAP = true: AA odd
// layout (plane qbar at x - c_q, through a wall plane q of the own cell).
// blockDim.x is a multiple of 32, so a warp never spans two lattice rows and
// lane 0 of a warp starts a 64-cell segment of its row.  Inactive lanes
// (x0 >= nx) read a valid pair and take part in the shuffles.
template <bool SWAP, typename T, typename R>
__device__ __forceinline__ void gather2(const T *grid, const Cell &c, const Geo &g, int lane, int x0, bool active,
                                        int own, R f0[Q], R f1[Q])
{
    const int xs = active ? x0 : 0;
    // Phase 1: issue every load before any shuffle (shuffles wait for their
    // operand, and interleaving them with the loads would serialise memory
    // latencies).  lo/hi: the own pair of the source row (or, through a y/z
    // wall, the own cell's reflected pair); e: the element beyond the warp's
    // edge for the +-x populations, loaded only by the edge lane.
    R lo[Q], hi[Q], e[Q];
    bool wyz[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cx = CX(q), cy = CY(q), cz = CZ(q);
        const int ys = cy == 0 ? c.y : (cy > 0 ? c.ym : c.yp);
        const int zs = cz == 0 ? c.z : (cz > 0 ? c.zm : c.zp);
        bool w = false;
        if (cy > 0) w |= c.bym;
        if (cy < 0) w |= c.byp;
        if (cz > 0) w |= c.bzm;
        if (cz < 0) w |= c.bzp;
        wyz[q] = w;
        const T *plane = grid + (long long)(SWAP ? OPP(q) : q) * g.ncell;   // streamed value
        const T *bplane = grid + (long long)(SWAP ? q : OPP(q)) * g.ncell;  // bounced value
        const int srow = zs * c.nxy + ys * c.nx;
        Pair<T>::load(w ? bplane + own + xs : plane + srow + xs, lo[q], hi[q]);
        e[q] = R(0);
        if (cx > 0) {  // pull from x - 1: lane 0 needs element x0 - 1
            const bool need = lane == 0 && active && !w;
            const T *a = (xs == 0 && g.wall_x) ? bplane + own + xs : plane + srow + (xs == 0 ? g.nx - 1 : xs - 1);
            if (need) e[q] = Storage<T>::load(a);
        } else if (cx < 0) {  // pull from x + 1: the last lane of a segment needs element x0 + 2
            const bool need = (lane == 31 || xs + 2 >= g.nx) && active && !w;
            const T *a = (xs + 2 >= g.nx && g.wall_x) ? bplane + own + xs + 1
                                                       : plane + srow + (xs + 2 >= g.nx ? 0 : xs + 2);
            if (need) e[q] = Storage<T>::load(a);
        }
    }
    // Phase 2: assemble the shifted pairs.
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cx = CX(q);
        if (cx == 0) {
            f0[q] = lo[q];
            f1[q] = hi[q];
        } else if (cx > 0) {
            R left = __shfl_up_sync(0xffffffffu, hi[q], 1);
            if (lane == 0) left = e[q];
            f0[q] = wyz[q] ? lo[q] : left;
            f1[q] = wyz[q] ? hi[q] : lo[q];
        } else {
            R right = __shfl_down_sync(0xffffffffu, lo[q], 1);
            if (lane == 31 || xs + 2 >= g.nx) right = e[q];
            f0[q] = wyz[q] ? lo[q] : hi[q];
            f1[q] = wyz[q] ? hi[q] : right;
        }
    }
}

// A/B pull step, two cells (x0, x0 + 1) per thread.
template <typename T, bool RHO0>
__global__ void __launch_bounds__(256) k_step_ab2(const T *__restrict__ src, T *__restrict__ dst, Geo g,
                                                  Relax<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    const int lane = threadIdx.x & 31;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (y >= g.ny) return;  // uniform across the warp
    const bool active = x0 < g.nx;
    Cell c(active ? x0 : 0, y, z, g);
    const int own = z * c.nxy + y * c.nx;
    R f0[Q], f1[Q];
    gather2<false>(src, c, g, lane, x0, active, own, f0, f1);
    if (!active) return;
    collide_lean<R, RHO0>(f0, p);
    collide_lean<R, RHO0>(f1, p);
#pragma unroll
    for (int q = 0; q < Q; ++q) Pair<T>::store(dst + (long long)q * g.ncell + own + x0, f0[q], f1[q]);
}

// AA odd step, two cells per thread: gather plane qbar from x - c_q (pairs,
// as above), collide, and write plane q at x + c_q.  A +-x shifted write is
// assembled into the aligned pair (x0, x0 + 1) of the target row from the own
// values and the neighbouring lane's (warp shuffle); the element that belongs
// to the neighbouring warp's pair is written by the edge lane as a scalar.
// Through a wall the value goes to plane qbar of the own cell.  Every
// location is written by exactly one thread, as in the one-cell kernel.
template <typename T, bool RHO0>
__global__ void __launch_bounds__(256, 2) k_step_aa_odd2(T *grid, Geo g, Relax<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    const int lane = threadIdx.x & 31;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (y >= g.ny) return;  // uniform across the warp
    const bool active = x0 < g.nx;
    Cell c(active ? x0 : 0, y, z, g);
    const int own = z * c.nxy + y * c.nx;
    R f0[Q], f1[Q];
    gather2<true>(grid, c, g, lane, x0, active, own, f0, f1);
    if (active) {
        collide_lean<R, RHO0>(f0, p);
        collide_lean<R, RHO0>(f1, p);
    }
    const bool last = lane == 31 || x0 + 2 >= g.nx;  // right edge of this warp's segment
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cx = CX(q), cy = CY(q), cz = CZ(q);
        const int yt = cy == 0 ? y : (cy > 0 ? c.yp : c.ym);
        const int zt = cz == 0 ? z : (cz > 0 ? c.zp : c.zm);
        bool w = false;
        if (cy > 0) w |= c.byp;
        if (cy < 0) w |= c.bym;
        if (cz > 0) w |= c.bzp;
        if (cz < 0) w |= c.bzm;
        T *plane = grid + (long long)q * g.ncell;        // streamed value
        T *bplane = grid + (long long)OPP(q) * g.ncell;  // bounced value
        const int trow = zt * c.nxy + yt * c.nx;
        if (cx == 0) {
            if (active) Pair<T>::store(w ? bplane + own + x0 : plane + trow + x0, f0[q], f1[q]);
        } else if (cx > 0) {
            // element x0 of the target row receives cell x0 - 1, element x0 + 1 cell x0
            const R left = __shfl_up_sync(0xffffffffu, f1[q], 1);
            if (!active) continue;
            if (w) {
                Pair<T>::store(bplane + own + x0, f0[q], f1[q]);
                continue;
            }
            if (lane == 0)
                Storage<T>::store(plane + trow + x0 + 1, f0[q]);
            else
                Pair<T>::store(plane + trow + x0, left, f0[q]);
            if (last) {  // cell x0 + 1 goes to x0 + 2: the next segment, the periodic image, or a wall
                if (x0 + 2 >= g.nx && g.wall_x)
                    Storage<T>::store(bplane + own + x0 + 1, f1[q]);
                else
                    Storage<T>::store(plane + trow + (x0 + 2 >= g.nx ? 0 : x0 + 2), f1[q]);
            }
        } else {
            // element x0 of the target row receives cell x0 + 1, element x0 + 1 cell x0 + 2
            const R right = __shfl_down_sync(0xffffffffu, f0[q], 1);
            if (!active) continue;
            if (w) {
                Pair<T>::store(bplane + own + x0, f0[q], f1[q]);
                continue;
            }
            if (last)
                Storage<T>::store(plane + trow + x0, f1[q]);
            else
                Pair<T>::store(plane + trow + x0, f1[q], right);
            if (lane == 0) {  // cell x0 goes to x0 - 1: the previous segment, the periodic image, or a wall
                if (x0 == 0 && g.wall_x)
                    Storage<T>::store(bplane + own + x0, f0[q]);
                else
                    Storage<T>::store(plane + trow + (x0 == 0 ? g.nx - 1 : x0 - 1), f0[q]);
            }
        }
    }
}

// AA in-place steps.  Even: own cell only (read q, write qbar).  Odd: read
// qbar at x - c_q, write q at x + c_q (bounce-back through walls stays in the
// own cell).  Every location is read and written by exactly one thread.
template <typename T, int ODD, bool RHO0>
__global__ void __launch_bounds__(256) k_step_aa(T *grid, Geo g, Relax<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    Cell c(x, y, z, g);
    R f[Q];
    if (ODD) {
        gather<AA_ODD>(grid, c, g.ncell, f);
        collide_lean<R, RHO0>(f, p);
        scatter<D_AA_ODD>(grid, c, g.ncell, f);
    } else {
        gather<AA_EVEN>(grid, c, g.ncell, f);
        collide_lean<R, RHO0>(f, p);
        scatter<D_AA_EVEN>(grid, c, g.ncell, f);
    }
}

// AA even step, two cells per thread: purely local, so every access is an
// aligned pair.
template <typename T, bool RHO0>
__global__ void __launch_bounds__(256) k_step_aa_even2(T *grid, Geo g, Relax<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x0 >= g.nx || y >= g.ny) return;
    const long long own = ((long long)z * g.ny + y) * g.nx + x0;
    R f0[Q], f1[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) Pair<T>::load(grid + (long long)q * g.ncell + own, f0[q], f1[q]);
    collide_lean<R, RHO0>(f0, p);
    collide_lean<R, RHO0>(f1, p);
#pragma unroll
    for (int q = 0; q < Q; ++q) Pair<T>::store(grid + (long long)OPP(q) * g.ncell + own, f0[q], f1[q]);
}

template <typename T, bool RHO0>
static cudaError_t step_t(int kind, const void *src, void *dst, const Geo &g, const CollBoth &cb, LaunchShape s,
                          cudaStream_t stream)
{
    using R = typename Storage<T>::R;
    Relax<R> p = to_relax<R>(cb);
    dim3 block(s.bx, s.by, 1);
    const bool pairs = s.cells_x == 2 && (g.nx % 2) == 0 && (s.bx % 32) == 0;
    const int span = pairs ? 2 * s.bx : s.bx;
    dim3 grid((g.nx + span - 1) / span, (g.ny + s.by - 1) / s.by, g.nz);
    if (kind == 0) {
        if (pairs)
            k_step_ab2<T, RHO0><<<grid, block, 0, stream>>>((const T *)src, (T *)dst, g, p);
        else
            k_step_ab<T, RHO0><<<grid, block, 0, stream>>>((const T *)src, (T *)dst, g, p);
    } else if (kind == 1) {
        if (pairs)
            k_step_aa_even2<T, RHO0><<<grid, block, 0, stream>>>((T *)dst, g, p);
        else
            k_step_aa<T, 0, RHO0><<<grid, block, 0, stream>>>((T *)dst, g, p);
    } else {
        if (pairs)
            k_step_aa_odd2<T, RHO0><<<grid, block, 0, stream>>>((T *)dst, g, p);
        else
            k_step_aa<T, 1, RHO0><<<grid, block, 0, stream>>>((T *)dst, g, p);
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t step_rho0(int kind, const void *src, void *dst, const Geo &g, const CollBoth &cb, LaunchShape s,
                            cudaStream_t stream)
{
    return cb.rho0_is_rho ? step_t<T, true>(kind, src, dst, g, cb, s, stream)
                          : step_t<T, false>(kind, src, dst, g, cb, s, stream);
}

cudaError_t launch_step(int prec, int kind, const void *src, void *dst, const Geo &g, const CollBoth &c,
                        LaunchShape s, cudaStream_t stream)
{
    switch (prec) {
    case P_F64: return step_rho0<double>(kind, src, dst, g, c, s, stream);
    case P_F32: return step_rho0<float>(kind, src, dst, g, c, s, stream);
    case P_F16: return step_rho0<__half>(kind, src, dst, g, c, s, stream);
    case P_BF16: return step_rho0<__nv_bfloat16>(kind, src, dst, g, c, s, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
