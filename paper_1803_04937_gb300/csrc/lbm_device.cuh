// Device-side building blocks of the D3Q19 library: the lattice, storage
// conversions, lattice geometry (periodic wrap and half-way bounce-back), the
// gather / scatter patterns of the A/B and AA propagation schemes, and the
// collision of Eq. 15 (SRT) or its TRT split, written in shifted variables
// g_q = f_q - w_q.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lbm_launch.h"

namespace lbm {

constexpr int Q = 19;

// D3Q19 velocity set of Sec. 2.3 in this library's order: q = 0 rest, then
// nine pairs (q, q+1) with c_{q+1} = -c_q: three faces, six edges.
__host__ __device__ constexpr int CX(int q)
{
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[q];
}
__host__ __device__ constexpr int CY(int q)
{
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[q];
}
__host__ __device__ constexpr int CZ(int q)
{
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[q];
}
__host__ __device__ constexpr int OPP(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ constexpr int NORM2(int q) { return CX(q) * CX(q) + CY(q) * CY(q) + CZ(q) * CZ(q); }
// weights 1/3, 1/18, 1/36 (Sec. 2.3)
template <typename R>
__host__ __device__ constexpr R WQ(int q)
{
    return NORM2(q) == 0 ? R(1) / R(3) : (NORM2(q) == 1 ? R(1) / R(18) : R(1) / R(36));
}

// ---------------------------------------------------------------- storage

template <typename T> struct Storage;
template <> struct Storage<double> {
    using R = double;
    static __device__ __forceinline__ R load(const double *p) { return *p; }
    static __device__ __forceinline__ void store(double *p, R v) { *p = v; }
};
template <> struct Storage<float> {
    using R = float;
    static __device__ __forceinline__ R load(const float *p) { return *p; }
    static __device__ __forceinline__ void store(float *p, R v) { *p = v; }
};
template <> struct Storage<__half> {
    using R = float;
    static __device__ __forceinline__ R load(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void store(__half *p, R v) { *p = __float2half_rn(v); }
};
template <> struct Storage<__nv_bfloat16> {
    using R = float;
    static __device__ __forceinline__ R load(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, R v) { *p = __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------- geometry

struct Geo {
    int nx, ny, nz;
    int wall_x, wall_y, wall_z;  // 1: half-way bounce-back walls at both ends
    long long ncell;             // plane stride of the SoA grid, nx * ny * nz
};

// One lattice cell with its wrapped neighbour coordinates and the wall flags
// of its six faces (true when the neighbour across that face is beyond a wall).
struct Cell {
    int x, y, z;
    int xm, xp, ym, yp, zm, zp;
    bool bxm, bxp, bym, byp, bzm, bzp;
    int nx, nxy;

    __device__ __forceinline__ Cell(int x_, int y_, int z_, const Geo &g) : x(x_), y(y_), z(z_)
    {
        xm = x == 0 ? g.nx - 1 : x - 1;
        xp = x == g.nx - 1 ? 0 : x + 1;
        ym = y == 0 ? g.ny - 1 : y - 1;
        yp = y == g.ny - 1 ? 0 : y + 1;
        zm = z == 0 ? g.nz - 1 : z - 1;
        zp = z == g.nz - 1 ? 0 : z + 1;
        bxm = g.wall_x && x == 0;
        bxp = g.wall_x && x == g.nx - 1;
        bym = g.wall_y && y == 0;
        byp = g.wall_y && y == g.ny - 1;
        bzm = g.wall_z && z == 0;
        bzp = g.wall_z && z == g.nz - 1;
        nx = g.nx;
        nxy = g.nx * g.ny;
    }
    __device__ __forceinline__ int self() const { return (z * nxy) + y * nx + x; }

    // Cell x + s*c_q (s = +1: push target, s = -1: pull source).  Sets
    // `wall` when the link crosses a bounce-back wall.
    template <int S>
    __device__ __forceinline__ int along(int q, bool &wall) const
    {
        const int cx = S * CX(q), cy = S * CY(q), cz = S * CZ(q);
        int xs = cx == 0 ? x : (cx > 0 ? xp : xm);
        int ys = cy == 0 ? y : (cy > 0 ? yp : ym);
        int zs = cz == 0 ? z : (cz > 0 ? zp : zm);
        bool w = false;
        if (cx > 0) w |= bxp;
        if (cx < 0) w |= bxm;
        if (cy > 0) w |= byp;
        if (cy < 0) w |= bym;
        if (cz > 0) w |= bzp;
        if (cz < 0) w |= bzm;
        wall = w;
        return zs * nxy + ys * nx + xs;
    }
};

// State layouts.  The canonical state is f_q(x, t) after streaming, before
// collision.  How it sits in memory:
//   AB      : grid[q][x - c_q] (the previous step's post-collision value that
//             streams into x); through a wall, grid[qbar][x].
//   AA_EVEN : grid[q][x] (after an even number of AA steps).
//   AA_ODD  : grid[qbar][x - c_q]; through a wall grid[q][x] (after an odd
//             number of AA steps).
enum Layout { AB = 0, AA_EVEN = 1, AA_ODD = 2 };

template <int L, typename T, typename R>
__device__ __forceinline__ void gather(const T *grid, const Cell &c, long long ncell, R g[Q])
{
    const int self = c.self();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        long long off;
        if (L == AA_EVEN) {
            off = (long long)q * ncell + self;
        } else {
            bool wall;
            int src = c.template along<-1>(q, wall);
            if (L == AB)
                off = wall ? (long long)OPP(q) * ncell + self : (long long)q * ncell + src;
            else
                off = wall ? (long long)q * ncell + self : (long long)OPP(q) * ncell + src;
        }
        g[q] = Storage<T>::load(grid + off);
    }
}

// Where post-collision values of a step go:
//   AB_NEXT : grid[q][x]                 (pull scheme, next step gathers them)
//   AA_EVEN : grid[qbar][x]
//   AA_ODD  : grid[q][x + c_q]; through a wall grid[qbar][x]
// and, to write a canonical state f_q(x) into a grid so that the AB gather
// returns it: AB_CANON : grid[q][x - c_q]; through a wall grid[qbar][x].
enum Dest { D_AB_NEXT = 0, D_AA_EVEN = 1, D_AA_ODD = 2, D_AB_CANON = 3 };

template <int D, typename T, typename R>
__device__ __forceinline__ void scatter(T *grid, const Cell &c, long long ncell, const R g[Q])
{
    const int self = c.self();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        long long off;
        if (D == D_AB_NEXT) {
            off = (long long)q * ncell + self;
        } else if (D == D_AA_EVEN) {
            off = (long long)OPP(q) * ncell + self;
        } else if (D == D_AA_ODD) {
            bool wall;
            int dst = c.template along<1>(q, wall);
            off = wall ? (long long)OPP(q) * ncell + self : (long long)q * ncell + dst;
        } else {
            bool wall;
            int dst = c.template along<-1>(q, wall);
            off = wall ? (long long)OPP(q) * ncell + self : (long long)q * ncell + dst;
        }
        Storage<T>::store(grid + off, g[q]);
    }
}

// ---------------------------------------------------------------- reductions

// Sum over the block (blockDim.x a multiple of 32, at most 1024 threads);
// the result is valid in thread 0.  Fixed order: deterministic.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    v = 0.0;
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

__device__ __forceinline__ double block_max(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    v = 0.0;
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    return v;
}

// ---------------------------------------------------------------- physics

// Per-launch collision constants (prepared on the host).
template <typename R>
struct Coll {
    R omega_p;        // 1 / tau
    R omega_m;        // 1 / tau-  (= omega_p for SRT)
    R kappa;          // 0: D3Q19-S (Eq. 14), 1: D3Q19-I (Eq. 22)
    R half_a[3];      // a / 2, the velocity shift of Eq. 17
    R force[9];       // (1 - omega_m / 2) F_q for the first member q = 2k+1 of pair k
    int rho0_is_rho;  // 0: rho0 = 1, 1: rho0 = rho
};

// Macroscopic quantities of the shifted populations: drho = rho - 1,
// u from rho0 u = j + a/2 (Eq. 16, Eq. 17), and rho0.
template <typename R>
static inline Coll<R> to_coll(const CollBoth &c)
{
    Coll<R> p;
    p.omega_p = R(c.omega_p);
    p.omega_m = R(c.omega_m);
    p.kappa = R(c.kappa);
    for (int i = 0; i < 3; ++i) p.half_a[i] = R(c.half_a[i]);
    for (int k = 0; k < 9; ++k) p.force[k] = R(c.force[k]);
    p.rho0_is_rho = c.rho0_is_rho;
    return p;
}

template <typename R>
__device__ __forceinline__ void macro(const R g[Q], const Coll<R> &p, R &drho, R &rho0, R u[3])
{
    R s = g[0];
    R jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        s += g[q];
        if (CX(q) > 0) jx += g[q];
        if (CX(q) < 0) jx -= g[q];
        if (CY(q) > 0) jy += g[q];
        if (CY(q) < 0) jy -= g[q];
        if (CZ(q) > 0) jz += g[q];
        if (CZ(q) < 0) jz -= g[q];
    }
    drho = s;
    rho0 = p.rho0_is_rho ? R(1) + s : R(1);
    R inv = p.rho0_is_rho ? R(1) / rho0 : R(1);
    u[0] = (jx + p.half_a[0]) * inv;
    u[1] = (jy + p.half_a[1]) * inv;
    u[2] = (jz + p.half_a[2]) * inv;
}

// Equilibrium of pair k (q = 2k+1 and its opposite) in shifted form:
//   geq_q = sym + asym,  geq_qbar = sym - asym,
// with the standard part w (drho + rho0 (9/2 (c.u)^2 - 3/2 u^2)), asym =
// 3 w rho0 c.u, plus kappa * rho0 * Delta_q where D3Q19-I = D3Q19-S + Delta:
//   face along axis a:   Delta = -(u^2 - u_a^2) / 12
//   edge in plane (a,b): Delta = u_c^2 / 24   (c the third axis)
// (the difference of Eq. 22 and Eq. 14 written per velocity group; both
// equilibria run the same instructions and differ only in kappa).
template <typename R, int q>
__device__ __forceinline__ void pair_equilibrium(const R u[3], R uu, R drho, R rho0, R kappa, R &sym, R &asym)
{
    constexpr int cx = CX(q), cy = CY(q), cz = CZ(q);
    const R w = WQ<R>(q);
    R cu = R(cx) * u[0] + R(cy) * u[1] + R(cz) * u[2];
    R delta;
    if (NORM2(q) == 1) {
        R ua = cx != 0 ? u[0] : (cy != 0 ? u[1] : u[2]);
        delta = (ua * ua - uu) * (R(1) / R(12));
    } else {
        R uc = cx == 0 ? u[0] : (cy == 0 ? u[1] : u[2]);
        delta = uc * uc * (R(1) / R(24));
    }
    sym = w * (drho + rho0 * (R(4.5) * cu * cu - R(1.5) * uu)) + kappa * rho0 * delta;
    asym = w * rho0 * R(3) * cu;
}

template <typename R>
__device__ __forceinline__ R rest_equilibrium(R uu, R drho, R rho0, R kappa)
{
    return WQ<R>(0) * (drho - rho0 * R(1.5) * uu) + kappa * rho0 * uu * (R(1) / R(6));
}

// Collision in place: g <- g - omega+ (g+ - geq+) - omega- (g- - geq-) +
// (1 - omega-/2) F_q.  For SRT omega- = omega+ and this is Eq. 15.
template <typename R, int k>
__device__ __forceinline__ void collide_pair(R g[Q], const R u[3], R uu, R drho, R rho0, const Coll<R> &p)
{
    constexpr int q = 2 * k + 1;
    R sym, asym;
    pair_equilibrium<R, q>(u, uu, drho, rho0, p.kappa, sym, asym);
    R gp = R(0.5) * (g[q] + g[q + 1]);
    R gm = R(0.5) * (g[q] - g[q + 1]);
    R a1 = p.omega_p * (gp - sym);
    R a2 = p.omega_m * (gm - asym);
    g[q] = g[q] - a1 - a2 + p.force[k];
    g[q + 1] = g[q + 1] - a1 + a2 - p.force[k];
}

template <typename R>
__device__ __forceinline__ void collide(R g[Q], const Coll<R> &p)
{
    R drho, rho0, u[3];
    macro(g, p, drho, rho0, u);
    R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    g[0] = g[0] - p.omega_p * (g[0] - rest_equilibrium(uu, drho, rho0, p.kappa));
    collide_pair<R, 0>(g, u, uu, drho, rho0, p);
    collide_pair<R, 1>(g, u, uu, drho, rho0, p);
    collide_pair<R, 2>(g, u, uu, drho, rho0, p);
    collide_pair<R, 3>(g, u, uu, drho, rho0, p);
    collide_pair<R, 4>(g, u, uu, drho, rho0, p);
    collide_pair<R, 5>(g, u, uu, drho, rho0, p);
    collide_pair<R, 6>(g, u, uu, drho, rho0, p);
    collide_pair<R, 7>(g, u, uu, drho, rho0, p);
    collide_pair<R, 8>(g, u, uu, drho, rho0, p);
}

// ---------------------------------------------------------------- lean collision (step kernels)

// Per-launch constants of the collision, folded so that a cell update needs
// few instructions.  With P = rho0 (1, or rho when rho0 = rho) and base =
// drho - 3/2 P u^2, the symmetric (even) equilibrium part of a pair is
//   faces along a:     wf base - kf u^2 + Kf u_a^2
//   edges normal to c: we base + ke u_c^2 + Ke (c.u)^2
//   rest:              w0 base + k0 u^2
// (kappa = 0: D3Q19-S; kappa = 1 adds the D3Q19-I corrections Delta), and the
// antisymmetric part is A/2 (c.u) with A = 6 w P.  The factors that carry P
// are stored for P = 1 and scaled per cell when rho0 = rho.
template <typename R>
struct Relax {
    R hp, hm, wp;    // omega+ / 2, omega- / 2, omega+
    R w0, wf, we;    // 1/3, 1/18, 1/36
    R k0, kf, ke;    // kappa / 6, kappa / 12, kappa / 24
    R Kf, Ke;        // 9/2 wf + kappa / 12, 9/2 we
    R Af, Ae;        // 6 wf, 6 we  (twice the antisymmetric coefficient)
    R half_a[3];     // a / 2
    R force[9];      // (1 - omega- / 2) F_q, q = 2k+1
    R hb, h4;        // MRT: (omega+ - omega_bulk) / 2, (omega+ - omega_4) / 2
};

template <typename R>
static inline Relax<R> to_relax(const CollBoth &c)
{
    const double wp = c.omega_p, wm = c.omega_m, k = c.kappa;
    const double w0 = 1.0 / 3.0, wf = 1.0 / 18.0, we = 1.0 / 36.0;
    Relax<R> r;
    r.hp = R(0.5 * wp);
    r.hm = R(0.5 * wm);
    r.wp = R(wp);
    r.w0 = R(w0);
    r.wf = R(wf);
    r.we = R(we);
    r.k0 = R(k / 6.0);
    r.kf = R(k / 12.0);
    r.ke = R(k / 24.0);
    r.Kf = R(4.5 * wf + k / 12.0);
    r.Ke = R(4.5 * we);
    // The equilibrium's first moment is (Af + 4 Ae) u per axis; with the
    // weights rounded to R it would be u (1 + eps), and the antisymmetric
    // relaxation would then grow the momentum by omega- eps every step (2000
    // FP32 steps: ~1e-4).  Af is chosen so that Af + 4 Ae = 1 exactly in R
    // (1 - 4 Ae is exact by Sterbenz's lemma).
    r.Ae = R(1.0 / 6.0);
    r.Af = R(1) - R(4) * r.Ae;
    for (int i = 0; i < 3; ++i) r.half_a[i] = R(c.half_a[i]);
    for (int i = 0; i < 9; ++i) r.force[i] = R(c.force[i]);
    r.hb = R(0.5 * (wp - c.omega_bulk));
    r.h4 = R(0.5 * (wp - c.omega_4));
    return r;
}

// Error-free sum (Knuth's TwoSum): hi + lo tracks hi + v exactly, hi holding
// the rounded sum and lo the accumulated rounding errors.
template <typename R>
__device__ __forceinline__ void two_sum_acc(R &hi, R &lo, R v)
{
    const R s = hi + v;
    const R bv = s - hi;
    lo += (hi - (s - bv)) + (v - bv);
    hi = s;
}

// Moments and symmetric-equilibrium bases of one cell, shared by the step and
// the adjoint.  s[k], d[k]: sum and difference of pair k (q = 2k+1, q + 1).
//
// COMP (rho0 = 1 only): the momentum is summed with TwoSum, and du = (j +
// a/2) - u, the part of the exact velocity that rounding u drops, is kept.
// The antisymmetric relaxation moves the momentum by -omega- (j + a/2 - u)
// per step (zero in exact arithmetic); with a rounded u, that is -omega- du
// every step, and in a flow that changes slowly (a channel accelerated from
// rest by a body force) these errors add up coherently: FP32 storage, 5000
// steps, 1x256x1 channel column in emulation: 1.9e-5 of max|u| against the
// FP64 oracle.  neq() subtracts du from the face pair of each axis, which
// makes the momentum balance exact again; what remains is the storage
// rounding (same emulation: 9e-7).
template <typename R, bool RHO0_IS_RHO, bool COMP = false>
struct CellEq {
    R s[9], d[9];
    R u[3], u2[3], uu, P;
    R du[3];
    R Bf, Be[3], eq0;
    R Kf, Ke, Af, Ae;

    __device__ __forceinline__ CellEq(const R g[Q], const Relax<R> &p)
    {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            s[k] = g[2 * k + 1] + g[2 * k + 2];
            d[k] = g[2 * k + 1] - g[2 * k + 2];
        }
        const R drho = g[0] + (((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])) + s[8]);
        R j[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int q = 2 * k + 1;
            if (CX(q) > 0) j[0] += d[k];
            if (CX(q) < 0) j[0] -= d[k];
            if (CY(q) > 0) j[1] += d[k];
            if (CY(q) < 0) j[1] -= d[k];
            if (CZ(q) > 0) j[2] += d[k];
            if (CZ(q) < 0) j[2] -= d[k];
        }
        P = R(1);
        if (RHO0_IS_RHO) {
            P = R(1) + drho;
            const R inv = R(1) / P;
#pragma unroll
            for (int i = 0; i < 3; ++i) u[i] = (j[i] + p.half_a[i]) * inv;
        } else if (COMP) {
            // pair k < 3 is the face pair of axis k (c = +e_k): it starts the sum
            R hi[3] = {d[0], d[1], d[2]}, lo[3] = {R(0), R(0), R(0)};
#pragma unroll
            for (int k = 3; k < 9; ++k) {
                const int q = 2 * k + 1;
                if (CX(q) != 0) two_sum_acc(hi[0], lo[0], CX(q) > 0 ? d[k] : -d[k]);
                if (CY(q) != 0) two_sum_acc(hi[1], lo[1], CY(q) > 0 ? d[k] : -d[k]);
                if (CZ(q) != 0) two_sum_acc(hi[2], lo[2], CZ(q) > 0 ? d[k] : -d[k]);
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                u[i] = hi[i];
                two_sum_acc(u[i], lo[i], p.half_a[i]);
                du[i] = lo[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < 3; ++i) u[i] = j[i] + p.half_a[i];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) u2[i] = u[i] * u[i];
        uu = u2[0] + u2[1] + u2[2];
        R k0 = p.k0, kf = p.kf, ke = p.ke;
        Kf = p.Kf;
        Ke = p.Ke;
        Af = p.Af;
        Ae = p.Ae;
        if (RHO0_IS_RHO) {
            k0 *= P; kf *= P; ke *= P; Kf *= P; Ke *= P; Af *= P; Ae *= P;
        }
        const R base = drho - R(1.5) * P * uu;
        Bf = p.wf * base - kf * uu;
#pragma unroll
        for (int i = 0; i < 3; ++i) Be[i] = p.we * base + ke * u2[i];
        eq0 = p.w0 * base + k0 * uu;
    }

    // Non-equilibrium parts of pair k: s - 2 sym and d - 2 asym, each formed
    // by one fused multiply-add so that only the small result is rounded.
    template <int k>
    __device__ __forceinline__ void neq(R &nsym, R &nasym) const
    {
        constexpr int q = 2 * k + 1;
        const R cu = R(CX(q)) * u[0] + R(CY(q)) * u[1] + R(CZ(q)) * u[2];
        R sym, A;
        if (NORM2(q) == 1) {
            const int a = CX(q) ? 0 : (CY(q) ? 1 : 2);
            sym = Bf + Kf * u2[a];
            A = Af;
        } else {
            const int c = CX(q) == 0 ? 0 : (CY(q) == 0 ? 1 : 2);
            sym = Be[c] + Ke * (cu * cu);
            A = Ae;
        }
        nsym = fma(R(-2), sym, s[k]);
        nasym = fma(-A, cu, d[k]);
        if constexpr (COMP && !RHO0_IS_RHO && k < 3) nasym -= du[k];
    }
};

// One collision (Eq. 15, or its TRT split) of the shifted populations g in
// place: g -/+ (omega+/2)(s - 2 sym) -/+ (omega-/2)(d - 2 asym) +/- (1 -
// omega-/2) F for the two members of each pair; the same result as the
// textbook form g - omega+ (g+ - geq+) - omega- (g- - geq-) + (1 - omega-/2) F
// up to rounding order.  With ONE_ROUNDING the change of each population is
// formed first by one fma (small numbers, small rounding) and added to g in one
// operation: one rounding at the scale of g instead of two (measured on the
// 256^3 FP32 shear wave after 2000 steps: worst error against the FP64 oracle
// 1.1e-5 -> 3.7e-6).  The step kernels take it for FP32 and FP64 storage
// (one_rounding_v); with 16-bit storage the rounding at the store is 2^13 times
// coarser than FP32's, so the two-rounding form loses nothing there, and some
// 16-bit kernels run it faster (walled channel 512x256x256, BF16: 77.8 -> 79.8
// GLUPS; D3Q27 four cells, FP16: 59.6 -> 62.9).
template <typename T>
constexpr bool one_rounding_v = sizeof(T) >= 4;

// FP32 storage (FP32 arithmetic with the one-rounding update) also sums the
// momentum with compensation (CellEq, COMP): 16-bit storage rounds far more
// coarsely at the store, and FP64 arithmetic does not need it.
template <typename R, bool ONE_ROUNDING>
constexpr bool compensated_v = ONE_ROUNDING && std::is_same<R, float>::value;

template <typename R, bool RHO0_IS_RHO, bool ONE_ROUNDING, int k>
__device__ __forceinline__ void relax_pair(R g[Q], const CellEq<R, RHO0_IS_RHO, compensated_v<R, ONE_ROUNDING>> &e,
                                           const Relax<R> &p)
{
    constexpr int q = 2 * k + 1;
    R nsym, nasym;
    e.template neq<k>(nsym, nasym);
    const R b = fma(p.hm, nasym, -p.force[k]);
    if (ONE_ROUNDING) {
        g[q] = g[q] - fma(p.hp, nsym, b);
        g[q + 1] = g[q + 1] - fma(p.hp, nsym, -b);
    } else {
        const R a1 = p.hp * nsym;
        g[q] = (g[q] - a1) - b;
        g[q + 1] = (g[q + 1] - a1) + b;
    }
}

template <typename R, bool RHO0_IS_RHO, bool ONE_ROUNDING>
__device__ __forceinline__ void collide_lean(R g[Q], const Relax<R> &p)
{
    const CellEq<R, RHO0_IS_RHO, compensated_v<R, ONE_ROUNDING>> e(g, p);
    g[0] = fma(-p.wp, g[0] - e.eq0, g[0]);
    relax_pair<R, RHO0_IS_RHO, ONE_ROUNDING, 0>(g, e, p);
    relax_pair<R, RHO0_IS_RHO, ONE_ROUNDING, 1>(g, e, p);
    relax_pair<R, RHO0_IS_RHO, ONE_ROUNDING, 2>(g, e, p);
    relax_pair<R, RHO0_IS_RHO, ONE_ROUNDING, 3>(g, e, p);
    relax_pair<R, RHO0_IS_RHO, ONE_ROUNDING, 4>(g, e, p);
    relax_pair<R, RHO0_IS_RHO, ONE_ROUNDING, 5>(g, e, p);
    relax_pair<R, RHO0_IS_RHO, ONE_ROUNDING, 6>(g, e, p);
    relax_pair<R, RHO0_IS_RHO, ONE_ROUNDING, 7>(g, e, p);
    relax_pair<R, RHO0_IS_RHO, ONE_ROUNDING, 8>(g, e, p);
}

// MRT collision (Sec. 3.2-3.3) in population space.  The even part of the
// non-equilibrium (rest n0 and pair sums ns) has, in the monomial moment basis,
// the second-order moments P and the fourth-order moments Q_c = sum over the
// two edge pairs normal to axis c (xi_a^2 xi_b^2, {a,b,c} = {x,y,z}); its
// zeroth moment is zero.  Relaxing the deviator of P at omega+, the trace
// T = tr P at omega_bulk and Q at omega_4 equals relaxing everything at
// omega+ and adding back (omega+ - omega_bulk) times the population vector
// whose only non-zero moment is that trace (rest -T, faces T/3, edges 0),
// plus (omega+ - omega_4) times the vector whose only non-zero moments are
// the Q (rest sum Q, face a Q_a - sum Q, edges normal to c Q_c/2); these are
// the columns of the inverse moment matrix for those moments.  The odd part
// relaxes at omega- with the force, exactly as in collide_lean.
template <typename R, bool RHO0_IS_RHO, bool ONE_ROUNDING>
__device__ __forceinline__ void collide_mrt(R g[Q], const Relax<R> &p)
{
    const CellEq<R, RHO0_IS_RHO, compensated_v<R, ONE_ROUNDING>> e(g, p);
    R ns[9], na[9];
    e.template neq<0>(ns[0], na[0]);
    e.template neq<1>(ns[1], na[1]);
    e.template neq<2>(ns[2], na[2]);
    e.template neq<3>(ns[3], na[3]);
    e.template neq<4>(ns[4], na[4]);
    e.template neq<5>(ns[5], na[5]);
    e.template neq<6>(ns[6], na[6]);
    e.template neq<7>(ns[7], na[7]);
    e.template neq<8>(ns[8], na[8]);
    R faces = R(0), Qn[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int q = 2 * k + 1;
        if (NORM2(q) == 1) faces += ns[k];
        else Qn[CX(q) == 0 ? 0 : (CY(q) == 0 ? 1 : 2)] += ns[k];
    }
    const R Qsum = (Qn[0] + Qn[1]) + Qn[2];
    const R T = fma(R(2), Qsum, faces);
    const R bT = p.hb * T;       // (omega+ - omega_bulk) T / 2
    const R bQ = p.h4 * Qsum;    // (omega+ - omega_4) sum Q / 2
    g[0] = fma(-p.wp, g[0] - e.eq0, g[0]) - R(2) * (bT - bQ);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int q = 2 * k + 1;
        R corr;  // (omega+ - omega_bulk) B / 2 + (omega+ - omega_4) G / 2 for this pair
        if (NORM2(q) == 1) {
            const int a = CX(q) ? 0 : (CY(q) ? 1 : 2);
            corr = fma(p.h4, Qn[a], bT * R(1.0 / 3.0) - bQ);
        } else {
            const int c = CX(q) == 0 ? 0 : (CY(q) == 0 ? 1 : 2);
            corr = R(0.5) * p.h4 * Qn[c];
        }
        const R a1 = fma(p.hp, ns[k], -corr);
        const R b = fma(p.hm, na[k], -p.force[k]);
        if (ONE_ROUNDING) {
            g[q] = g[q] - (a1 + b);
            g[q + 1] = g[q + 1] - (a1 - b);
        } else {
            g[q] = (g[q] - a1) - b;
            g[q + 1] = (g[q + 1] - a1) + b;
        }
    }
}

// Step collision: the lean SRT/TRT update, or MRT.
template <typename R, bool RHO0_IS_RHO, bool MRT, bool ONE_ROUNDING>
__device__ __forceinline__ void collide_any(R g[Q], const Relax<R> &p)
{
    if constexpr (MRT)
        collide_mrt<R, RHO0_IS_RHO, ONE_ROUNDING>(g, p);
    else
        collide_lean<R, RHO0_IS_RHO, ONE_ROUNDING>(g, p);
}

// Shifted equilibrium geq_q = feq_q(rho, u) - w_q for all q (lbm_init).
template <typename R>
__device__ __forceinline__ void equilibrium_all(R rho, const R u[3], const Coll<R> &p, R g[Q])
{
    R drho = rho - R(1);
    R rho0 = p.rho0_is_rho ? rho : R(1);
    R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    g[0] = rest_equilibrium(uu, drho, rho0, p.kappa);
#define LBM_EQ_PAIR(k)                                                              \
    {                                                                               \
        R s_, a_;                                                                   \
        pair_equilibrium<R, 2 * k + 1>(u, uu, drho, rho0, p.kappa, s_, a_);         \
        g[2 * k + 1] = s_ + a_;                                                     \
        g[2 * k + 2] = s_ - a_;                                                     \
    }
    LBM_EQ_PAIR(0) LBM_EQ_PAIR(1) LBM_EQ_PAIR(2) LBM_EQ_PAIR(3) LBM_EQ_PAIR(4)
    LBM_EQ_PAIR(5) LBM_EQ_PAIR(6) LBM_EQ_PAIR(7) LBM_EQ_PAIR(8)
#undef LBM_EQ_PAIR
}

}  // namespace lbm
