// Fused stream + collide time step (Eq. 15; D3Q19-S / D3Q19-I equilibria;
// SRT / TRT; periodic or half-way bounce-back; Buick-Greated force): kernel
// templates, instantiated per storage precision in lbm_step_<prec>.cu.
//
// Each thread gathers the populations that stream into its cell(s), collides
// them in registers (FP32, or FP64 for FP64 storage) and stores the
// post-collision values.  Structure-of-arrays storage gives coalesced accesses
// along x for every population.  Algorithmic traffic: 19 loads + 19 stores
// per cell.
//
// Address arithmetic is kept to one 32-bit index per access: the base pointer
// of each population plane comes from the kernel parameters (a table of 19
// pointers) and the nine source/target row offsets (y +- 1, z +- 1, wrapped)
// are formed once per thread.  WALLS = false compiles the periodic lattice
// without any bounce-back logic.
//
// Three thread mappings:
//  - one cell per thread (any nx; the FP32 and FP64 default): scalar loads;
//    the +-x populations are read one element off alignment, which L1/L2
//    absorb without extra DRAM traffic.
//  - two neighbouring cells per thread (nx even): every population is read
//    and written as an aligned pair (half2 / bfloat162 / float2 / double2);
//    a +-x shifted pair is assembled from the own pair and one element of the
//    neighbouring lane's pair (warp shuffle), with one scalar access at the
//    warp's edge.
//  - four cells per thread (16-bit storage, nx % 4 == 0; the 16-bit default):
//    8-byte quads of raw 16-bit codes; a +-x shifted window is formed from the
//    aligned quad and its aligned neighbour quad by funnel shifts (load4w).
#pragma once

#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace lbm {

template <typename T> struct Planes {
    T *p[Q];
};

template <typename T>
static inline Planes<T> planes_of(void *base, long long ncell)
{
    Planes<T> r;
    for (int q = 0; q < Q; ++q) r.p[q] = (T *)base + (long long)q * ncell;
    return r;
}

// The rows an A/B launch covers: y in [y0, y1), z in [z0, z0 + gridDim.z).
// The four-cell step on a lattice with walls on y and/or z runs its interior
// rows, whose links cross no wall, through the periodic kernel and only the
// wall rows through the walled one (split_rows).
struct Rows {
    int y0, y1, z0;
};

// Per-thread lattice geometry: wrapped neighbour coordinates, the nine row
// offsets of the rows y + dy, z + dz (dy, dz in {-1, 0, 1}) and, with walls,
// the wall flags of the six faces of the cell(s).
template <bool WALLS>
struct Site {
    int x, xm, xp;      // x and its wrapped neighbours (first cell of the thread)
    int row[3][3];      // row[dy + 1][dz + 1] = ((z + dz) ny + (y + dy)) nx, wrapped
    int own;            // row[1][1]
    bool bxm, bxp, bym, byp, bzm, bzp;

    __device__ __forceinline__ Site(int x_, int y, int z, int span, const Geo &g)
    {
        x = x_;
        xm = x == 0 ? g.nx - 1 : x - 1;
        xp = x + span >= g.nx ? x + span - g.nx : x + span;  // first cell after the thread's span
        const int ym = y == 0 ? g.ny - 1 : y - 1;
        const int yp = y == g.ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? g.nz - 1 : z - 1;
        const int zp = z == g.nz - 1 ? 0 : z + 1;
        const int nxy = g.nx * g.ny;
        const int ys[3] = {ym, y, yp}, zs[3] = {zm, z, zp};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) row[a][b] = zs[b] * nxy + ys[a] * g.nx;
        own = row[1][1];
        if (WALLS) {
            bxm = g.wall_x && x == 0;
            bxp = g.wall_x && x + span >= g.nx;
            bym = g.wall_y && y == 0;
            byp = g.wall_y && y == g.ny - 1;
            bzm = g.wall_z && z == 0;
            bzp = g.wall_z && z == g.nz - 1;
        } else {
            bxm = bxp = bym = byp = bzm = bzp = false;
        }
    }

    // Does the link from the cell along s * c_q cross a y/z wall?
    template <int S>
    __device__ __forceinline__ bool wall_yz(int q) const
    {
        if (!WALLS) return false;
        const int cy = S * CY(q), cz = S * CZ(q);
        bool w = false;
        if (cy > 0) w |= byp;
        if (cy < 0) w |= bym;
        if (cz > 0) w |= bzp;
        if (cz < 0) w |= bzm;
        return w;
    }
    template <int S>
    __device__ __forceinline__ int row_along(int q) const
    {
        return row[S * CY(q) + 1][S * CZ(q) + 1];
    }
};

// Rows that touch no y/z wall on a lattice with walls on x (XONLY kernels):
// the y/z wall flags are constant false, so only the x-wall selects remain.
template <bool XONLY, bool WALLS>
__device__ __forceinline__ void drop_yz(Site<WALLS> &s)
{
    if constexpr (XONLY) s.bym = s.byp = s.bzm = s.bzp = false;
}

// An in-place step writes the locations it has read; left alone, the compiler
// keeps the 19 load addresses (64-bit each) alive through the collisions to
// reuse them for the stores, and spills.  Passing the offsets through an
// empty asm statement hides that equality, so the store addresses are formed
// again from the kernel-parameter base pointers after the collisions.
__device__ __forceinline__ void opaque(int &v) { asm volatile("" : "+r"(v)); }
template <bool WALLS>
__device__ __forceinline__ void opaque(Site<WALLS> &s)
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) opaque(s.row[a][b]);
    opaque(s.own);
    opaque(s.x);
    opaque(s.xm);
    opaque(s.xp);
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

// ---------------------------------------------------------------- one cell per thread

// Gather of the populations streaming into one cell.  SWAP = false: A/B
// layout (plane q at x - c_q; through a wall, plane qbar of the own cell);
// SWAP = true: AA odd layout (plane qbar at x - c_q; through a wall, plane q
// of the own cell).
template <bool SWAP, bool WALLS, typename T, typename R>
__device__ __forceinline__ void gather1(const Planes<T> &P, const Site<WALLS> &s, R f[Q])
{
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cx = CX(q);
        const int xs = cx == 0 ? s.x : (cx > 0 ? s.xm : s.xp);
        bool w = s.template wall_yz<-1>(q);
        if (WALLS) {
            if (cx > 0) w |= s.bxm;
            if (cx < 0) w |= s.bxp;
        }
        const T *src = SWAP ? P.p[OPP(q)] : P.p[q];
        const T *bnc = SWAP ? P.p[q] : P.p[OPP(q)];
        const T *a = w ? bnc + s.own + s.x : src + s.template row_along<-1>(q) + xs;
        f[q] = Storage<T>::load(a);
    }
}

// Gather, collision and stores of k_ab1 for one cell.
template <typename T, bool RHO0, bool WALLS, bool MRT>
__device__ __forceinline__ void ab1_body(const Planes<T> &src, const Planes<T> &dst, const Site<WALLS> &s,
                                         const Relax<typename Storage<T>::R> &p)
{
    using R = typename Storage<T>::R;
    R f[Q];
    gather1<false>(src, s, f);
    collide_any<R, RHO0, MRT, one_rounding_v<T>>(f, p);
#pragma unroll
    for (int q = 0; q < Q; ++q) Storage<T>::store(dst.p[q] + s.own + s.x, f[q]);
}

template <typename T, bool RHO0, bool WALLS, bool MRT = false>
__global__ void __launch_bounds__(256) k_ab1(Planes<T> src, Planes<T> dst, Geo g, Relax<typename Storage<T>::R> p,
                                             Rows r)
{
    using R = typename Storage<T>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = r.y0 + (int)(blockIdx.y * blockDim.y + threadIdx.y);
    const int z = r.z0 + (int)blockIdx.z;
    if (x >= g.nx || y >= r.y1) return;
    if constexpr (WALLS) {
        // warps with no cell at a wall take the periodic body (uniform branch per warp)
        const Site<true> sw(x, y, z, 1, g);
        const bool touches = sw.bxm || sw.bxp || sw.bym || sw.byp || sw.bzm || sw.bzp;
        if (__any_sync(__activemask(), touches)) {
            ab1_body<T, RHO0, true, MRT>(src, dst, sw, p);
            return;
        }
    }
    ab1_body<T, RHO0, false, MRT>(src, dst, Site<false>(x, y, z, 1, g), p);
}

// Blocks per SM the one-cell AA steps are compiled for.  With the compensated
// momentum sum of FP32 storage the compiler's own choice for the odd step is
// 94 registers, two blocks of 256 threads per SM (FP32 AA pair 0.98 -> 0.83
// of the copy bandwidth at 256^3).  Measured for the FP32 SRT/TRT pair
// (even, odd blocks; 256^3 / 768^3): (5, 3) 0.932 / 0.943 (odd step 80
// registers, 16 bytes spilled; even 48, none), (6, 3) 0.911 / 0.924, (5, 2)
// 0.889 / 0.897, (6, 4) 0.859 / 0.871; (5, 3) is kept.
template <typename T, bool MRT>
constexpr int aa1_blocks(bool odd)
{
    return (std::is_same<T, float>::value && !MRT) ? (odd ? 3 : 5) : 1;
}

// AA even step: own cell only (read plane q, write plane qbar).  The store
// side takes its own copy of the plane table (the same pointers): given one
// table, the compiler keeps its 19 pointers in registers between the loads and
// the stores (80 instead of 40 registers; +1.5 % FP32, +2.8 % FP64 measured).
template <typename T, bool RHO0, bool MRT = false>
__global__ void __launch_bounds__(256, aa1_blocks<T, MRT>(false)) k_aa_even1(Planes<T> P, Planes<T> Pw, Geo g,
                                                                           Relax<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int own = (z * g.ny + y) * g.nx + x;
    R f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = Storage<T>::load(P.p[q] + own);
    collide_any<R, RHO0, MRT, one_rounding_v<T>>(f, p);
#pragma unroll
    for (int q = 0; q < Q; ++q) Storage<T>::store(Pw.p[OPP(q)] + own, f[q]);
}

// AA odd step: read plane qbar at x - c_q, write plane q at x + c_q (through
// a wall: read plane q / write plane qbar of the own cell).  Every location is
// read and written by exactly one thread.
template <typename T, bool RHO0, bool WALLS, bool MRT = false, bool ROWS = false, bool XONLY = false>
__global__ void __launch_bounds__(256, aa1_blocks<T, MRT>(true)) k_aa_odd1(Planes<T> P, Geo g,
                                                                         Relax<typename Storage<T>::R> p, Rows r)
{
    using R = typename Storage<T>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = (ROWS ? r.y0 : 0) + (int)(blockIdx.y * blockDim.y + threadIdx.y);
    const int z = (ROWS ? r.z0 : 0) + (int)blockIdx.z;
    if (x >= g.nx || y >= (ROWS ? r.y1 : g.ny)) return;
    Site<WALLS> s(x, y, z, 1, g);
    drop_yz<XONLY>(s);
    R f[Q];
    gather1<true>(P, s, f);
    collide_any<R, RHO0, MRT, one_rounding_v<T>>(f, p);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cx = CX(q);
        const int xt = cx == 0 ? x : (cx > 0 ? s.xp : s.xm);
        bool w = s.template wall_yz<1>(q);
        if (WALLS) {
            if (cx > 0) w |= s.bxp;
            if (cx < 0) w |= s.bxm;
        }
        T *a = w ? P.p[OPP(q)] + s.own + x : P.p[q] + s.template row_along<1>(q) + xt;
        Storage<T>::store(a, f[q]);
    }
}

// ---------------------------------------------------------------- two cells per thread

// Pair-wise gather for the cells (x0, x0 + 1), x0 even, nx even (layouts as
// in gather1).  blockDim.x is a multiple of 32, so a warp never spans two
// lattice rows and lane 0 of a warp starts a 64-cell segment of its row.
// Inactive lanes (x0 >= nx) read a valid pair and take part in the shuffles.
template <bool SWAP, bool WALLS, typename T, typename R>
__device__ __forceinline__ void gather2(const Planes<T> &P, const Site<WALLS> &s, const Geo &g, int lane,
                                        bool active, R f0[Q], R f1[Q])
{
    const int x0 = s.x;
    const bool last = lane == 31 || x0 + 2 >= g.nx;
    // Phase 1: issue every load before any shuffle.  lo/hi: the own pair of
    // the source row (or, through a y/z wall, the own cell's reflected pair);
    // e: the element beyond the segment's edge for the +-x populations.
    R lo[Q], hi[Q], e[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cx = CX(q);
        const bool w = s.template wall_yz<-1>(q);
        const T *src = SWAP ? P.p[OPP(q)] : P.p[q];
        const T *bnc = SWAP ? P.p[q] : P.p[OPP(q)];
        const int srow = s.template row_along<-1>(q);
        Pair<T>::load(w ? bnc + s.own + x0 : src + srow + x0, lo[q], hi[q]);
        e[q] = R(0);
        if (cx > 0) {  // pull from x - 1: lane 0 needs element x0 - 1
            const T *a = (WALLS && s.bxm) ? bnc + s.own + x0 : src + srow + s.xm;
            if (lane == 0 && active && !w) e[q] = Storage<T>::load(a);
        } else if (cx < 0) {  // pull from x + 1: the segment's last lane needs element x0 + 2
            const T *a = (WALLS && s.bxp) ? bnc + s.own + x0 + 1 : src + srow + s.xp;
            if (last && active && !w) e[q] = Storage<T>::load(a);
        }
    }
    // Phase 2: assemble the shifted pairs.
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cx = CX(q);
        const bool w = s.template wall_yz<-1>(q);
        if (cx == 0) {
            f0[q] = lo[q];
            f1[q] = hi[q];
        } else if (cx > 0) {
            R left = __shfl_up_sync(0xffffffffu, hi[q], 1);
            if (lane == 0) left = e[q];
            f0[q] = w ? lo[q] : left;
            f1[q] = w ? hi[q] : lo[q];
        } else {
            R right = __shfl_down_sync(0xffffffffu, lo[q], 1);
            if (last) right = e[q];
            f0[q] = w ? lo[q] : hi[q];
            f1[q] = w ? hi[q] : right;
        }
    }
}

template <typename T, bool RHO0, bool WALLS>
__global__ void __launch_bounds__(256, 4) k_ab2(Planes<T> src, Planes<T> dst, Geo g, Relax<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    const int lane = threadIdx.x & 31;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (y >= g.ny) return;  // uniform across the warp
    const bool active = x0 < g.nx;
    const Site<WALLS> s(active ? x0 : 0, y, z, 2, g);
    R f0[Q], f1[Q];
    gather2<false>(src, s, g, lane, active, f0, f1);
    if (!active) return;
    collide_lean<R, RHO0, one_rounding_v<T>>(f0, p);
    collide_lean<R, RHO0, one_rounding_v<T>>(f1, p);
#pragma unroll
    for (int q = 0; q < Q; ++q) Pair<T>::store(dst.p[q] + s.own + x0, f0[q], f1[q]);
}

template <typename T, bool RHO0>
__global__ void __launch_bounds__(256) k_aa_even2(Planes<T> P, Geo g, Relax<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x0 >= g.nx || y >= g.ny) return;
    const int own = (z * g.ny + y) * g.nx + x0;
    R f0[Q], f1[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) Pair<T>::load(P.p[q] + own, f0[q], f1[q]);
    collide_lean<R, RHO0, one_rounding_v<T>>(f0, p);
    collide_lean<R, RHO0, one_rounding_v<T>>(f1, p);
#pragma unroll
    for (int q = 0; q < Q; ++q) Pair<T>::store(P.p[OPP(q)] + own, f0[q], f1[q]);
}

// AA odd step, two cells per thread: gather plane qbar from x - c_q (pairs),
// collide, and write plane q at x + c_q.  A +-x shifted write is assembled
// into the aligned pair (x0, x0 + 1) of the target row from the own values and
// the neighbouring lane's (warp shuffle); the element that belongs to the
// neighbouring segment is written by the edge lane as a scalar.  Through a
// wall the value goes to plane qbar of the own cell.  Every location is
// written by exactly one thread, as in the one-cell kernel.
template <typename T, bool RHO0, bool WALLS>
__global__ void __launch_bounds__(256, 2) k_aa_odd2(Planes<T> P, Geo g, Relax<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    const int lane = threadIdx.x & 31;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (y >= g.ny) return;  // uniform across the warp
    const bool active = x0 < g.nx;
    const Site<WALLS> s(active ? x0 : 0, y, z, 2, g);
    R f0[Q], f1[Q];
    gather2<true>(P, s, g, lane, active, f0, f1);
    if (active) {
        collide_lean<R, RHO0, one_rounding_v<T>>(f0, p);
        collide_lean<R, RHO0, one_rounding_v<T>>(f1, p);
    }
    const bool last = lane == 31 || x0 + 2 >= g.nx;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cx = CX(q);
        const bool w = s.template wall_yz<1>(q);
        T *dst = P.p[q];
        T *bnc = P.p[OPP(q)];
        const int trow = s.template row_along<1>(q);
        if (cx == 0) {
            if (active) Pair<T>::store(w ? bnc + s.own + x0 : dst + trow + x0, f0[q], f1[q]);
        } else if (cx > 0) {
            // element x0 of the target row receives cell x0 - 1, element x0 + 1 cell x0
            const R left = __shfl_up_sync(0xffffffffu, f1[q], 1);
            if (!active) continue;
            if (w) {
                Pair<T>::store(bnc + s.own + x0, f0[q], f1[q]);
                continue;
            }
            if (lane == 0)
                Storage<T>::store(dst + trow + x0 + 1, f0[q]);
            else
                Pair<T>::store(dst + trow + x0, left, f0[q]);
            if (last)  // cell x0 + 1 goes to x0 + 2: the next segment, the periodic image, or a wall
                Storage<T>::store((WALLS && s.bxp) ? bnc + s.own + x0 + 1 : dst + trow + s.xp, f1[q]);
        } else {
            // element x0 of the target row receives cell x0 + 1, element x0 + 1 cell x0 + 2
            const R right = __shfl_down_sync(0xffffffffu, f0[q], 1);
            if (!active) continue;
            if (w) {
                Pair<T>::store(bnc + s.own + x0, f0[q], f1[q]);
                continue;
            }
            if (last)
                Storage<T>::store(dst + trow + x0, f1[q]);
            else
                Pair<T>::store(dst + trow + x0, f1[q], right);
            if (lane == 0)  // cell x0 goes to x0 - 1: the previous segment, the periodic image, or a wall
                Storage<T>::store((WALLS && s.bxm) ? bnc + s.own + x0 : dst + trow + s.xm, f0[q]);
        }
    }
}

// ---------------------------------------------------------------- four cells per thread (16-bit storage)

// Raw 16-bit codes <-> float for the 16-bit storage types.
template <typename T> struct Bits16;
template <> struct Bits16<__half> {
    static __device__ __forceinline__ float to_float(unsigned int b)
    {
        return __half2float(__ushort_as_half((unsigned short)b));
    }
    static __device__ __forceinline__ unsigned int from_float(float v)
    {
        return __half_as_ushort(__float2half_rn(v));
    }
};
template <> struct Bits16<__nv_bfloat16> {
    static __device__ __forceinline__ float to_float(unsigned int b)
    {
        return __bfloat162float(__ushort_as_bfloat16((unsigned short)b));
    }
    static __device__ __forceinline__ unsigned int from_float(float v)
    {
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
};

// Element c (0..3) of four 16-bit codes packed in a uint2, and its replacement.
template <int c>
__device__ __forceinline__ unsigned int quad_get(const uint2 &v)
{
    const unsigned int w = c < 2 ? v.x : v.y;
    return (c & 1) ? (w >> 16) : (w & 0xffffu);
}
template <int c>
__device__ __forceinline__ void quad_set(uint2 &v, unsigned int b)
{
    unsigned int &w = c < 2 ? v.x : v.y;
    w = (c & 1) ? ((w & 0x0000ffffu) | (b << 16)) : ((w & 0xffff0000u) | (b & 0xffffu));
}

// Phase 1, windowed: for every population the four inputs of the cells
// x0 .. x0 + 3 as one 8-byte window of raw 16-bit codes.  A +-x shifted
// window is assembled from the aligned quad and its aligned neighbour quad
// (x0 - 4 or x0 + 4, wrapped) by two funnel shifts, so no lane needs another
// lane's data; the neighbour quads are the lines the adjacent lanes load
// anyway (L1 hits; no extra DRAM traffic).  Through a y/z wall the window is
// the own cells' reflected quad; at an x wall the element beyond the wall is
// the own cell's reflected slot.  SWAP as in load4.
template <bool SWAP, bool WALLS, typename T>
__device__ __forceinline__ void load4w(const Planes<T> &P, const Site<WALLS> &s, const Geo &g, uint2 (&win)[Q])
{
    const int xs = s.x;
    const int xprev = xs == 0 ? g.nx - 4 : xs - 4;
    const int xnext = xs + 4 >= g.nx ? 0 : xs + 4;
    uint2 nb[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cx = CX(q);
        const bool w = s.template wall_yz<-1>(q);
        const unsigned short *srcq = reinterpret_cast<const unsigned short *>(SWAP ? P.p[OPP(q)] : P.p[q]);
        const unsigned short *bncq = reinterpret_cast<const unsigned short *>(SWAP ? P.p[q] : P.p[OPP(q)]);
        const int srow = s.template row_along<-1>(q);
        const uint2 *pq = reinterpret_cast<const uint2 *>(w ? bncq + s.own + xs : srcq + srow + xs);
        const uint2 *pn = reinterpret_cast<const uint2 *>(srcq + srow + (cx > 0 ? xprev : xnext));
        const bool xwall = WALLS && ((cx > 0 && s.bxm) || (cx < 0 && s.bxp));
        if (xwall && !w) pn = reinterpret_cast<const uint2 *>(bncq + s.own + xs);
        // Non-coherent loads, also in the in-place AA odd step (SWAP): the
        // elements it uses of a quad are its own cells' inputs, which only this
        // thread writes, and only after it has read them; the other elements of
        // a neighbour quad may be stale there and are not used.
        win[q] = __ldg(pq);
        if (cx != 0) nb[q] = w ? make_uint2(0u, 0u) : __ldg(pn);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cx = CX(q);
        const bool w = s.template wall_yz<-1>(q);
        if (cx == 0 || w) continue;
        const uint2 c = win[q];
        uint2 n = nb[q];
        if (cx > 0) {
            // [x0 - 1, x0, x0 + 1, x0 + 2]: element 3 of the quad before (or the reflected x0)
            if (WALLS && s.bxm) n.y = n.x << 16;
            win[q].x = __funnelshift_l(n.y, c.x, 16);
            win[q].y = __funnelshift_l(c.x, c.y, 16);
        } else {
            // [x0 + 1, x0 + 2, x0 + 3, x0 + 4]: element 0 of the quad after (or the reflected x0 + 3)
            if (WALLS && s.bxp) n.x = n.y >> 16;
            win[q].x = __funnelshift_r(c.x, c.y, 16);
            win[q].y = __funnelshift_r(c.y, n.x, 16);
        }
    }
}

// Four collisions on windows: element c of every population's window is the
// input of cell c, and its result is written back into element c.
template <typename T, bool RHO0, bool MRT = false>
__device__ __forceinline__ void collide4(uint2 (&win)[Q], const Relax<float> &p)
{
#define LBM_AB4_CELL(c)                                                                      \
    {                                                                                        \
        float f[Q];                                                                          \
        _Pragma("unroll") for (int q = 0; q < Q; ++q) f[q] = Bits16<T>::to_float(quad_get<c>(win[q]));   \
        collide_any<float, RHO0, MRT, false>(f, p);                                          \
        _Pragma("unroll") for (int q = 0; q < Q; ++q) quad_set<c>(win[q], Bits16<T>::from_float(f[q]));  \
    }
    LBM_AB4_CELL(0) LBM_AB4_CELL(1) LBM_AB4_CELL(2) LBM_AB4_CELL(3)
#undef LBM_AB4_CELL
}

// A/B pull step for 16-bit storage, four cells (x0 .. x0 + 3) per thread,
// x0 a multiple of 4, nx a multiple of 4: every population is read and
// written as 8-byte quads, so the address work is shared by four cells.  The
// shifted inputs come from the aligned quad and its aligned neighbour by
// funnel shifts (load4w), so no lane waits for another; the four results are
// written back into the windows in place.  Replacing the earlier gather
// (neighbour elements by warp shuffles and a carry chain through the four
// cells) took this step from 0.88 to 1.04 of the measured copy bandwidth.
// Bitwise the same results as the one- and two-cell kernels.
// Loads, four collisions and stores of k_ab4 for one thread's quad.
template <typename T, bool RHO0, bool WALLS, bool MRT>
__device__ __forceinline__ void ab4_body(const Planes<T> &src, const Planes<T> &dst, const Site<WALLS> &s,
                                         const Geo &g, const Relax<float> &p)
{
    uint2 win[Q];
    load4w<false>(src, s, g, win);
    collide4<T, RHO0, MRT>(win, p);
#pragma unroll
    for (int q = 0; q < Q; ++q)
        *reinterpret_cast<uint2 *>(reinterpret_cast<unsigned short *>(dst.p[q]) + s.own + s.x) = win[q];
}

// Resident blocks per SM for k_ab4.  The walled FP16 kernel (both code paths
// inlined) spills at five blocks and runs faster at four with no spills; the
// walled BF16 kernel is the other way round (measured with the walled channel
// 512x256x256 as one walled launch: FP16 82.9 -> 84.5 GLUPS at four, BF16
// 79.9 -> 74.4).  With split_rows the walled kernel runs only the wall rows,
// or whole lattices with walls on x.
template <typename T, bool WALLS>
constexpr int ab4_blocks = (WALLS && std::is_same_v<T, __half>) ? 4 : 5;

// XONLY: rows that touch no y/z wall on a lattice with walls on x (a
// cavity's interior rows): one body with the x-wall selects only, which cost
// little (the end quads' shifted windows take the reflected own quad).
template <typename T, bool RHO0, bool WALLS, bool MRT = false, bool XONLY = false>
__global__ void __launch_bounds__(128, ab4_blocks<T, WALLS && !XONLY>) k_ab4(Planes<T> src, Planes<T> dst, Geo g,
                                                                              Relax<float> p, Rows r)
{
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = r.y0 + (int)(blockIdx.y * blockDim.y + threadIdx.y);
    const int z = r.z0 + (int)blockIdx.z;
    if (y >= r.y1 || x0 >= g.nx) return;  // no lane needs another lane's data
    if constexpr (XONLY) {
        Site<true> sx(x0, y, z, 4, g);
        drop_yz<true>(sx);
        ab4_body<T, RHO0, true, MRT>(src, dst, sx, g, p);
        return;
    }
    if constexpr (WALLS) {
        // A warp covers one row segment; where none of its cells touches a wall
        // (all but the wall rows and the row ends) it takes the periodic body,
        // which has no bounce-back selects.  The branch is uniform per warp.
        const Site<true> sw(x0, y, z, 4, g);
        const bool touches = sw.bxm || sw.bxp || sw.bym || sw.byp || sw.bzm || sw.bzp;
        if (__any_sync(__activemask(), touches)) {
            ab4_body<T, RHO0, true, MRT>(src, dst, sw, g, p);
            return;
        }
    }
    ab4_body<T, RHO0, false, MRT>(src, dst, Site<false>(x0, y, z, 4, g), g, p);
}

// AA even step for 16-bit storage, four cells per thread: own quads of plane
// q in, own quads of plane qbar out.  The stores take their own copy of the
// plane table (see k_aa_even1), which lets the step run five blocks per SM
// without spills (96 registers; with one table it needed 128).
template <typename T, bool RHO0, bool MRT = false>
__global__ void __launch_bounds__(128, 5) k_aa_even4(Planes<T> P, Planes<T> Pw, Geo g, Relax<float> p)
{
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x0 >= g.nx || y >= g.ny) return;
    const int own = (z * g.ny + y) * g.nx + x0;
    uint2 quad[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q)
        quad[q] = *reinterpret_cast<const uint2 *>(reinterpret_cast<const unsigned short *>(P.p[q]) + own);
    collide4<T, RHO0, MRT>(quad, p);
    int own_w = own;
    opaque(own_w);
#pragma unroll
    for (int q = 0; q < Q; ++q)
        *reinterpret_cast<uint2 *>(reinterpret_cast<unsigned short *>(Pw.p[OPP(q)]) + own_w) = quad[q];
}

// AA odd step for 16-bit storage, four cells per thread: gather plane qbar
// from x - c_q (as k_ab4 with the planes swapped), collide, and write plane q
// at x + c_q.  A +-x shifted write is assembled into the aligned quad
// (x0 .. x0 + 3) of the target row from three own results and one of the
// neighbouring lane (warp shuffle); at a segment's edge the lane writes the
// three own elements of the aligned quad and the edge lane writes the fourth
// result as a scalar into the neighbouring segment (or its periodic image, or
// through an x wall into plane qbar of the own cell).  Through a y/z wall the
// quad goes to plane qbar of the own cells.  Each location is written by one
// thread, and read (for a value that is used) only by that thread, as in the
// one-cell kernel.
template <typename T, bool RHO0, bool WALLS, bool MRT = false, bool ROWS = false, bool XONLY = false>
__global__ void __launch_bounds__(128, MRT ? 4 : 5) k_aa_odd4(Planes<T> P, Geo g, Relax<float> p, Rows r)
{
    const int lane = threadIdx.x & 31;
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = (ROWS ? r.y0 : 0) + (int)(blockIdx.y * blockDim.y + threadIdx.y);
    const int z = (ROWS ? r.z0 : 0) + (int)blockIdx.z;
    if (y >= (ROWS ? r.y1 : g.ny)) return;  // uniform across the warp
    const bool active = x0 < g.nx;
    Site<WALLS> s(active ? x0 : 0, y, z, 4, g);
    drop_yz<XONLY>(s);
    const int xs = s.x;
    const bool last = lane == 31 || xs + 4 >= g.nx;
    uint2 quad[Q];
    load4w<true>(P, s, g, quad);
    if (active) collide4<T, RHO0, MRT>(quad, p);
    Site<WALLS> sw = s;
    opaque(sw);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cx = CX(q);
        const bool w = s.template wall_yz<1>(q);
        unsigned short *dst = reinterpret_cast<unsigned short *>(P.p[q]);
        unsigned short *bnc = reinterpret_cast<unsigned short *>(P.p[OPP(q)]);
        const int trow = sw.template row_along<1>(q);
        if (cx == 0) {
            if (active) *reinterpret_cast<uint2 *>(w ? bnc + sw.own + sw.x : dst + trow + sw.x) = quad[q];
        } else if (cx > 0) {
            // target elements x0 .. x0 + 3 receive cells x0 - 1 .. x0 + 2
            const unsigned int left = __shfl_up_sync(0xffffffffu, quad[q].y >> 16, 1);
            if (!active) continue;
            if (w) {
                *reinterpret_cast<uint2 *>(bnc + sw.own + sw.x) = quad[q];
                continue;
            }
            unsigned short *t = dst + trow + sw.x;
            if (lane == 0) {  // element x0 belongs to the previous segment's last cell
                t[1] = (unsigned short)(quad[q].x & 0xffffu);
                *reinterpret_cast<unsigned int *>(t + 2) = __byte_perm(quad[q].x, quad[q].y, 0x5432);
            } else {
                uint2 v;
                v.x = __byte_perm(left, quad[q].x, 0x5410);
                v.y = __byte_perm(quad[q].x, quad[q].y, 0x5432);
                *reinterpret_cast<uint2 *>(t) = v;
            }
            if (last)  // cell x0 + 3 goes to x0 + 4: the next segment, the periodic image, or a wall
                *((WALLS && s.bxp) ? bnc + sw.own + sw.x + 3 : dst + trow + sw.xp) = (unsigned short)(quad[q].y >> 16);
        } else {
            // target elements x0 .. x0 + 3 receive cells x0 + 1 .. x0 + 4
            const unsigned int rgt = __shfl_down_sync(0xffffffffu, quad[q].x & 0xffffu, 1);
            if (!active) continue;
            if (w) {
                *reinterpret_cast<uint2 *>(bnc + sw.own + sw.x) = quad[q];
                continue;
            }
            unsigned short *t = dst + trow + sw.x;
            if (last) {  // element x0 + 3 belongs to the next segment's first cell
                *reinterpret_cast<unsigned int *>(t) = __byte_perm(quad[q].x, quad[q].y, 0x5432);
                t[2] = (unsigned short)(quad[q].y >> 16);
            } else {
                uint2 v;
                v.x = __byte_perm(quad[q].x, quad[q].y, 0x5432);
                v.y = __byte_perm(quad[q].y, rgt, 0x5432);
                *reinterpret_cast<uint2 *>(t) = v;
            }
            if (lane == 0)  // cell x0 goes to x0 - 1: the previous segment, the periodic image, or a wall
                *((WALLS && s.bxm) ? bnc + sw.own + sw.x : dst + trow + sw.xm) = (unsigned short)(quad[q].x & 0xffffu);
        }
    }
}

// ---------------------------------------------------------------- dispatch

// Calls launch(kind, rows, nz_rows) for the launches of one step.  A periodic
// lattice is one ROWS_PERIODIC launch over all rows.  With walls, the interior
// rows (no link crosses a y or z wall) run the periodic kernel, or with walls
// on x the kernel that has the x-wall selects only (ROWS_XWALLS), and the wall
// rows the walled one (ROWS_WALLED): rows y = 0 and ny - 1 over all z, then
// planes z = 0 and nz - 1 over the interior y; every row is in exactly one
// launch.  All kernels compute a cell with the same code as the single walled
// launch, so the results are bitwise the same.  The walled four-cell kernel
// carries both bodies and spills; keeping it to the wall rows took the walled
// channel 512x256x256 from 84.3 to 89.1 GLUPS (FP16) and from 80.0 to 86.9
// (BF16), and a cavity (walls on x, y and z) 512x256x256 from 0.76 to 0.95 of
// the copy bandwidth (FP16 A/B).
// Kinds of the launches of split_rows.
enum { ROWS_PERIODIC = 0, ROWS_WALLED = 1, ROWS_XWALLS = 2 };

template <bool WALLS, typename F>
static void split_rows(const Geo &g, F &&launch)
{
    if (!WALLS) {
        launch(ROWS_PERIODIC, Rows{0, g.ny, 0}, g.nz);
        return;
    }
    const int inner = g.wall_x ? ROWS_XWALLS : ROWS_PERIODIC;
    const int ylo = g.wall_y ? 1 : 0, yhi = g.wall_y ? g.ny - 1 : g.ny;
    const int zlo = g.wall_z ? 1 : 0, zhi = g.wall_z ? g.nz - 1 : g.nz;
    if (yhi > ylo && zhi > zlo) launch(inner, Rows{ylo, yhi, zlo}, zhi - zlo);
    if (g.wall_y) {
        launch(ROWS_WALLED, Rows{0, 1, 0}, g.nz);
        if (g.ny > 1) launch(ROWS_WALLED, Rows{g.ny - 1, g.ny, 0}, g.nz);
    }
    if (g.wall_z && yhi > ylo) {
        launch(ROWS_WALLED, Rows{ylo, yhi, 0}, 1);
        if (g.nz > 1) launch(ROWS_WALLED, Rows{ylo, yhi, g.nz - 1}, 1);
    }
}

// The one-cell A/B step stays one launch over all rows: its walled kernel
// already runs at the periodic kernel's speed (walled channel 512x256x256,
// FP32: 45.2 GLUPS as one launch, 44.8 split).
template <typename T, bool RHO0, bool WALLS, bool MRT>
static void launch_ab1(const Planes<T> &S, const Planes<T> &D, const Geo &g, const Relax<typename Storage<T>::R> &p,
                       dim3 block, cudaStream_t stream)
{
    const dim3 grid((g.nx + block.x - 1) / block.x, (g.ny + block.y - 1) / block.y, g.nz);
    k_ab1<T, RHO0, WALLS, MRT><<<grid, block, 0, stream>>>(S, D, g, p, Rows{0, g.ny, 0});
}

// The one-cell AA odd step, split into interior and wall rows like the
// four-cell one (walled channel 512x256x256, FP32: odd step 0.72 of the copy
// bandwidth as one walled launch).
template <typename T, bool RHO0, bool WALLS, bool MRT>
static void launch_aa_odd1(const Planes<T> &P, const Geo &g, const Relax<typename Storage<T>::R> &p, dim3 block,
                           cudaStream_t stream)
{
    split_rows<WALLS>(g, [&](int kind, Rows r, int nzr) {
        const dim3 grid((g.nx + block.x - 1) / block.x, (r.y1 - r.y0 + block.y - 1) / block.y, nzr);
        if (kind == ROWS_WALLED)
            k_aa_odd1<T, RHO0, true, MRT, WALLS><<<grid, block, 0, stream>>>(P, g, p, r);
        else if (kind == ROWS_XWALLS)
            k_aa_odd1<T, RHO0, true, MRT, true, true><<<grid, block, 0, stream>>>(P, g, p, r);
        else
            k_aa_odd1<T, RHO0, false, MRT, WALLS><<<grid, block, 0, stream>>>(P, g, p, r);
    });
}

template <typename T, bool RHO0, bool WALLS, bool MRT>
static void launch_ab4(const Planes<T> &S, const Planes<T> &D, const Geo &g, const Relax<float> &p, dim3 block4,
                       cudaStream_t stream)
{
    split_rows<WALLS>(g, [&](int kind, Rows r, int nzr) {
        const dim3 grid((g.nx + 4 * block4.x - 1) / (4 * block4.x), (r.y1 - r.y0 + block4.y - 1) / block4.y, nzr);
        if (kind == ROWS_WALLED)
            k_ab4<T, RHO0, true, MRT><<<grid, block4, 0, stream>>>(S, D, g, p, r);
        else if (kind == ROWS_XWALLS)
            k_ab4<T, RHO0, true, MRT, true><<<grid, block4, 0, stream>>>(S, D, g, p, r);
        else
            k_ab4<T, RHO0, false, MRT><<<grid, block4, 0, stream>>>(S, D, g, p, r);
    });
}

// The four-cell AA odd step, split into interior and wall rows as the A/B
// step is (split_rows): the walled kernel spills and runs the walled channel
// 512x256x256's odd step at 0.55 of the copy bandwidth (FP16 and BF16) as one
// launch.  Each location is read and written by one cell's thread only, so
// the launches may run in any order.
template <typename T, bool RHO0, bool WALLS, bool MRT>
static void launch_aa_odd4(const Planes<T> &P, const Geo &g, const Relax<float> &p, dim3 block4, cudaStream_t stream)
{
    split_rows<WALLS>(g, [&](int kind, Rows r, int nzr) {
        const dim3 grid((g.nx + 4 * block4.x - 1) / (4 * block4.x), (r.y1 - r.y0 + block4.y - 1) / block4.y, nzr);
        // the interior rows of a walled lattice take the x-walls-only kernel also
        // without x walls (its x flags are then false): it compiles to a faster
        // step than the periodic kernel with a row range (walled channel, FP16 AA
        // pair 0.81 -> 0.85, BF16 0.80 -> 0.82)
        if (kind == ROWS_WALLED)
            k_aa_odd4<T, RHO0, true, MRT, WALLS><<<grid, block4, 0, stream>>>(P, g, p, r);
        else if (WALLS)
            k_aa_odd4<T, RHO0, true, MRT, true, true><<<grid, block4, 0, stream>>>(P, g, p, r);
        else
            k_aa_odd4<T, RHO0, false, MRT><<<grid, block4, 0, stream>>>(P, g, p, r);
    });
}

template <typename T, bool RHO0, bool WALLS>
static cudaError_t step_t(int kind, void *src, void *dst, const Geo &g, const CollBoth &cb, LaunchShape ls,
                          cudaStream_t stream)
{
    using R = typename Storage<T>::R;
    const Relax<R> p = to_relax<R>(cb);
    const dim3 block(ls.bx, ls.by, 1);
    const bool quads = sizeof(T) == 2 && ls.cells_x == 4 && (g.nx % 4) == 0;
    if (cb.mrt && !quads) {
        // MRT: one cell per thread (16-bit storage with nx % 4 == 0 takes the four-cell kernels below)
        const dim3 grid1((g.nx + ls.bx - 1) / ls.bx, (g.ny + ls.by - 1) / ls.by, g.nz);
        const Planes<T> D = planes_of<T>(dst, g.ncell);
        if (kind == 0)
            launch_ab1<T, RHO0, WALLS, true>(planes_of<T>(src, g.ncell), D, g, p, block, stream);
        else if (kind == 1)
            k_aa_even1<T, RHO0, true><<<grid1, block, 0, stream>>>(D, D, g, p);
        else
            launch_aa_odd1<T, RHO0, WALLS, true>(D, g, p, block, stream);
        return cudaGetLastError();
    }
    const bool pairs = !quads && ls.cells_x >= 2 && (g.nx % 2) == 0 && (ls.bx % 32) == 0;
    if (quads) {
        // 128 threads; bx in {128, 64, 32} along x (whole warps per row segment), the
        // rest along y; bx leaves the fewest idle lanes at the end of a row (nx = 768:
        // 64, so three blocks cover the 192 quads of a row instead of two with 64
        // idle lanes), the larger on ties
        const int nq = g.nx / 4;
        int bx = 128, idle = (nq + 127) / 128 * 128 - nq;
        for (int c = 64; c >= 32; c /= 2) {
            const int w = (nq + c - 1) / c * c - nq;
            if (w < idle) {
                bx = c;
                idle = w;
            }
        }
        const dim3 block4(bx, 128 / bx, 1);
        const dim3 grid4((g.nx + 4 * bx - 1) / (4 * bx), (g.ny + block4.y - 1) / block4.y, g.nz);
        if constexpr (sizeof(T) == 2) {
            const Planes<T> D = planes_of<T>(dst, g.ncell);
            if (cb.mrt) {
                if (kind == 0)
                    launch_ab4<T, RHO0, WALLS, true>(planes_of<T>(src, g.ncell), D, g, p, block4, stream);
                else if (kind == 1)
                    k_aa_even4<T, RHO0, true><<<grid4, block4, 0, stream>>>(D, D, g, p);
                else
                    launch_aa_odd4<T, RHO0, WALLS, true>(D, g, p, block4, stream);
            } else if (kind == 0) {
                launch_ab4<T, RHO0, WALLS, false>(planes_of<T>(src, g.ncell), D, g, p, block4, stream);
            } else if (kind == 1) {
                k_aa_even4<T, RHO0><<<grid4, block4, 0, stream>>>(D, D, g, p);
            } else {
                launch_aa_odd4<T, RHO0, WALLS, false>(D, g, p, block4, stream);
            }
        }
        return cudaGetLastError();
    }
    const int span = pairs ? 2 * ls.bx : ls.bx;
    const dim3 grid((g.nx + span - 1) / span, (g.ny + ls.by - 1) / ls.by, g.nz);
    const Planes<T> D = planes_of<T>(dst, g.ncell);
    if (kind == 0) {
        const Planes<T> S = planes_of<T>(src, g.ncell);
        if (pairs)
            k_ab2<T, RHO0, WALLS><<<grid, block, 0, stream>>>(S, D, g, p);
        else
            launch_ab1<T, RHO0, WALLS, false>(S, D, g, p, block, stream);
    } else if (kind == 1) {
        if (pairs)
            k_aa_even2<T, RHO0><<<grid, block, 0, stream>>>(D, g, p);
        else
            k_aa_even1<T, RHO0><<<grid, block, 0, stream>>>(D, D, g, p);
    } else {
        if (pairs)
            k_aa_odd2<T, RHO0, WALLS><<<grid, block, 0, stream>>>(D, g, p);
        else
            launch_aa_odd1<T, RHO0, WALLS, false>(D, g, p, block, stream);
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t step_any(int kind, void *src, void *dst, const Geo &g, const CollBoth &cb, LaunchShape s,
                            cudaStream_t stream)
{
    const bool walls = g.wall_x || g.wall_y || g.wall_z;
    if (cb.rho0_is_rho)
        return walls ? step_t<T, true, true>(kind, src, dst, g, cb, s, stream)
                     : step_t<T, true, false>(kind, src, dst, g, cb, s, stream);
    return walls ? step_t<T, false, true>(kind, src, dst, g, cb, s, stream)
                 : step_t<T, false, false>(kind, src, dst, g, cb, s, stream);
}

}  // namespace lbm
