// D3Q27 stream + collide (Sec. 2.3 lattice; on D3Q27 the moment-matching
// construction of Sec. 3.1 gives the standard equilibrium of Eq. 14, so both
// equilibrium choices run Eq. 14), for the paper's D3Q19 / D3Q27 comparison:
// the same A/B pull scheme, force, TRT, boundaries and storage precisions as
// the D3Q19 path, with 27 loads + 27 stores per cell.  One cell per thread,
// or four for 16-bit storage.
//
// Also: initialisation f = feq(rho, u), moments and canonical copies for
// D3Q27 lattices.  (Reductions, AA and the adjoint are D3Q19 only.)
#include <cmath>

#include "lbm_step.cuh"

namespace lbm {
namespace q27 {

constexpr int Q27 = 27;

// This library's D3Q27 order: rest, then 13 pairs (q, q + 1) with
// c_{q+1} = -c_q: 3 faces, 6 edges, 4 corners.
__host__ __device__ constexpr int CX(int q)
{
    constexpr int t[Q27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
    return t[q];
}
__host__ __device__ constexpr int CY(int q)
{
    constexpr int t[Q27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, -1, 1, -1, 1};
    return t[q];
}
__host__ __device__ constexpr int CZ(int q)
{
    constexpr int t[Q27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[q];
}
__host__ __device__ constexpr int OPP(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ constexpr int NORM2(int q) { return CX(q) * CX(q) + CY(q) * CY(q) + CZ(q) * CZ(q); }
__host__ __device__ constexpr double WQ(int q)
{
    return NORM2(q) == 0 ? 8.0 / 27.0 : (NORM2(q) == 1 ? 2.0 / 27.0 : (NORM2(q) == 2 ? 1.0 / 54.0 : 1.0 / 216.0));
}

// Per-launch constants.  The antisymmetric equilibrium of a pair is
// (A_k / 2) c.u with A = 6 w; per axis the first moment is A_face + 4 A_edge +
// 4 A_corner = 1, and the constants are chosen so that this holds exactly in
// the working precision (no systematic momentum drift).
template <typename R>
struct Relax27 {
    R hp, hm, wp;
    R w[4];    // rest, face, edge, corner
    R K[4];    // 9/2 w
    R A[4];    // 6 w (A[0] unused)
    R half_a[3];
    R force[13];
};

template <typename R>
static inline Relax27<R> to_relax27(const CollBoth &c)
{
    Relax27<R> r;
    r.hp = R(0.5 * c.omega_p);
    r.hm = R(0.5 * c.omega_m);
    r.wp = R(c.omega_p);
    const double w[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
    for (int i = 0; i < 4; ++i) {
        r.w[i] = R(w[i]);
        r.K[i] = R(4.5 * w[i]);
    }
    // A_edge = R(1/9); A_corner rounded to a multiple of ulp(A_edge) / 4 so
    // that 1 - 4 A_edge - 4 A_corner is exactly representable in R.
    // (In FP32: ulp(1/9) = 2^-27, and 1 - 4 A_edge - 4 A_corner is a multiple
    // of 2^-25 in [1/4, 1/2), exact in FP32 and computed exactly in double.
    // In FP64 the residual is at the 1e-16 level.)
    double ae = 1.0 / 9.0, ac = 1.0 / 36.0;
    if (sizeof(R) == 4) {
        ae = (double)(float)(1.0 / 9.0);
        ac = std::round((1.0 / 36.0) * 134217728.0) / 134217728.0;  // multiple of 2^-27
    }
    r.A[0] = R(0);
    r.A[2] = R(ae);
    r.A[3] = R(ac);
    r.A[1] = R(1.0 - 4.0 * ae - 4.0 * ac);
    for (int i = 0; i < 3; ++i) r.half_a[i] = R(c.half_a[i]);
    const double wm = c.omega_m;
    for (int k = 0; k < 13; ++k) {
        const int q = 2 * k + 1;
        const double ca = CX(q) * 2.0 * c.half_a[0] + CY(q) * 2.0 * c.half_a[1] + CZ(q) * 2.0 * c.half_a[2];
        r.force[k] = R((1.0 - 0.5 * wm) * 3.0 * WQ(q) * ca);
    }
    return r;
}

// ONE_ROUNDING adds each population's change to g in one rounding, as the
// D3Q19 collision (relax_pair) does for FP32 and FP64 storage.
template <typename R, bool RHO0, bool ONE_ROUNDING>
__device__ __forceinline__ void collide27(R g[Q27], const Relax27<R> &p)
{
    R s[13], d[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        s[k] = g[2 * k + 1] + g[2 * k + 2];
        d[k] = g[2 * k + 1] - g[2 * k + 2];
    }
    R drho = g[0];
#pragma unroll
    for (int k = 0; k < 13; ++k) drho += s[k];
    R j[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        const int q = 2 * k + 1;
        if (CX(q)) j[0] += R(CX(q)) * d[k];
        if (CY(q)) j[1] += R(CY(q)) * d[k];
        if (CZ(q)) j[2] += R(CZ(q)) * d[k];
    }
    R P = R(1), u[3], du[3] = {R(0), R(0), R(0)};
    constexpr bool COMP = compensated_v<R, ONE_ROUNDING> && !RHO0;
    if (RHO0) {
        P = R(1) + drho;
        const R inv = R(1) / P;
#pragma unroll
        for (int i = 0; i < 3; ++i) u[i] = (j[i] + p.half_a[i]) * inv;
    } else if (COMP) {
        // compensated momentum, as CellEq does for D3Q19 (FP32 storage): u is
        // rounded, du = (j + a/2) - u exactly, and the face pair of each axis
        // (k = 0, 1, 2: c = +e_x, +e_y, +e_z) takes du out of its
        // antisymmetric non-equilibrium, so the momentum balance stays exact
        R hi[3] = {d[0], d[1], d[2]}, lo[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int k = 3; k < 13; ++k) {
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
    const R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const R base = drho - R(1.5) * P * uu;
    g[0] = fma(-p.wp, g[0] - p.w[0] * base, g[0]);
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        const int q = 2 * k + 1;
        const int cls = NORM2(q);
        const R cu = R(CX(q)) * u[0] + R(CY(q)) * u[1] + R(CZ(q)) * u[2];
        const R sym = p.w[cls] * base + (P * p.K[cls]) * (cu * cu);
        const R nsym = fma(R(-2), sym, s[k]);
        R nasym = fma(-(P * p.A[cls]), cu, d[k]);
        if (COMP && k < 3) nasym -= du[k];
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
}

// A/B pull step, one cell per thread.
template <typename T, bool RHO0, bool WALLS>
__global__ void __launch_bounds__(256) k27_ab1(const T *__restrict__ src, T *__restrict__ dst, Geo g,
                                               Relax27<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const Site<WALLS> s(x, y, z, 1, g);
    R f[Q27];
#pragma unroll
    for (int q = 0; q < Q27; ++q) {
        const int cx = CX(q), cy = CY(q), cz = CZ(q);
        const int xs = cx == 0 ? x : (cx > 0 ? s.xm : s.xp);
        bool w = false;
        if (WALLS) {
            if (cx > 0) w |= s.bxm;
            if (cx < 0) w |= s.bxp;
            if (cy > 0) w |= s.bym;
            if (cy < 0) w |= s.byp;
            if (cz > 0) w |= s.bzm;
            if (cz < 0) w |= s.bzp;
        }
        const long long a = w ? (long long)OPP(q) * g.ncell + s.own + x
                              : (long long)q * g.ncell + s.row[1 - cy][1 - cz] + xs;
        f[q] = Storage<T>::load(src + a);
    }
    collide27<R, RHO0, one_rounding_v<T>>(f, p);
#pragma unroll
    for (int q = 0; q < Q27; ++q) Storage<T>::store(dst + (long long)q * g.ncell + s.own + x, f[q]);
}

// A/B pull step for 16-bit storage, four cells per thread (nx % 4 == 0): the
// same windowed quads as the D3Q19 four-cell step (each +-x shifted window
// formed by funnel shifts from the aligned quad and its aligned neighbour),
// 27 populations.  Bitwise the same results as k27_ab1.  ROWS: only the rows
// y in [r.y0, r.y1), z in [r.z0, r.z0 + gridDim.z) (split_rows).
template <typename T, bool RHO0, bool WALLS, bool ROWS = false, bool XONLY = false>
__global__ void __launch_bounds__(128, 4) k27_ab4(const T *__restrict__ src, T *__restrict__ dst, Geo g,
                                                  Relax27<float> p, Rows r)
{
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = (ROWS ? r.y0 : 0) + (int)(blockIdx.y * blockDim.y + threadIdx.y);
    const int z = (ROWS ? r.z0 : 0) + (int)blockIdx.z;
    if (y >= (ROWS ? r.y1 : g.ny) || x0 >= g.nx) return;
    Site<WALLS> s(x0, y, z, 4, g);
    drop_yz<XONLY>(s);
    const int xprev = x0 == 0 ? g.nx - 4 : x0 - 4;
    const int xnext = x0 + 4 >= g.nx ? 0 : x0 + 4;
    const unsigned short *base = reinterpret_cast<const unsigned short *>(src);
    uint2 win[Q27], nb[Q27];
#pragma unroll
    for (int q = 0; q < Q27; ++q) {
        const int cx = CX(q), cy = CY(q), cz = CZ(q);
        bool w = false;
        if (WALLS) {
            if (cy > 0) w |= s.bym;
            if (cy < 0) w |= s.byp;
            if (cz > 0) w |= s.bzm;
            if (cz < 0) w |= s.bzp;
        }
        const unsigned short *plane = base + (long long)q * g.ncell + s.row[1 - cy][1 - cz];
        const unsigned short *bnc = base + (long long)OPP(q) * g.ncell + s.own;
        const uint2 *pq = reinterpret_cast<const uint2 *>(w ? bnc + x0 : plane + x0);
        const uint2 *pn = reinterpret_cast<const uint2 *>(plane + (cx > 0 ? xprev : xnext));
        const bool xwall = WALLS && ((cx > 0 && s.bxm) || (cx < 0 && s.bxp));
        if (xwall && !w) pn = reinterpret_cast<const uint2 *>(bnc + x0);
        win[q] = __ldg(pq);
        if (cx != 0) nb[q] = w ? make_uint2(0u, 0u) : __ldg(pn);
    }
#pragma unroll
    for (int q = 0; q < Q27; ++q) {
        const int cx = CX(q), cy = CY(q), cz = CZ(q);
        bool w = false;
        if (WALLS) {
            if (cy > 0) w |= s.bym;
            if (cy < 0) w |= s.byp;
            if (cz > 0) w |= s.bzm;
            if (cz < 0) w |= s.bzp;
        }
        if (cx == 0 || w) continue;
        const uint2 c = win[q];
        uint2 n = nb[q];
        if (cx > 0) {
            if (WALLS && s.bxm) n.y = n.x << 16;
            win[q].x = __funnelshift_l(n.y, c.x, 16);
            win[q].y = __funnelshift_l(c.x, c.y, 16);
        } else {
            if (WALLS && s.bxp) n.x = n.y >> 16;
            win[q].x = __funnelshift_r(c.x, c.y, 16);
            win[q].y = __funnelshift_r(c.y, n.x, 16);
        }
    }
#define LBM_AB27_CELL(c)                                                                     \
    {                                                                                        \
        float f[Q27];                                                                        \
        _Pragma("unroll") for (int q = 0; q < Q27; ++q) f[q] = Bits16<T>::to_float(quad_get<c>(win[q]));   \
        collide27<float, RHO0, false>(f, p);                                                 \
        _Pragma("unroll") for (int q = 0; q < Q27; ++q) quad_set<c>(win[q], Bits16<T>::from_float(f[q]));  \
    }
    LBM_AB27_CELL(0) LBM_AB27_CELL(1) LBM_AB27_CELL(2) LBM_AB27_CELL(3)
#undef LBM_AB27_CELL
    unsigned short *out = reinterpret_cast<unsigned short *>(dst);
#pragma unroll
    for (int q = 0; q < Q27; ++q)
        *reinterpret_cast<uint2 *>(out + (long long)q * g.ncell + s.own + x0) = win[q];
}

// Writes the canonical populations fc (f_q(x) - w_q) of cell x into an A/B
// grid so that the pull gather returns them: plane q at x - c_q, or through a
// wall plane qbar of x.
template <typename T, bool WALLS>
__device__ __forceinline__ void put_canonical(T *grid, const Site<WALLS> &s, int x, const Geo &g,
                                              const typename Storage<T>::R fc[Q27])
{
#pragma unroll
    for (int q = 0; q < Q27; ++q) {
        const int cx = CX(q), cy = CY(q), cz = CZ(q);
        const int xs = cx == 0 ? x : (cx > 0 ? s.xm : s.xp);
        bool w = false;
        if (WALLS) {
            if (cx > 0) w |= s.bxm;
            if (cx < 0) w |= s.bxp;
            if (cy > 0) w |= s.bym;
            if (cy < 0) w |= s.byp;
            if (cz > 0) w |= s.bzm;
            if (cz < 0) w |= s.bzp;
        }
        const long long a = w ? (long long)OPP(q) * g.ncell + s.own + x
                              : (long long)q * g.ncell + s.row[1 - cy][1 - cz] + xs;
        Storage<T>::store(grid + a, fc[q]);
    }
}

template <typename T, bool WALLS>
__device__ __forceinline__ void get_canonical(const T *grid, const Site<WALLS> &s, int x, const Geo &g,
                                              typename Storage<T>::R fc[Q27])
{
#pragma unroll
    for (int q = 0; q < Q27; ++q) {
        const int cx = CX(q), cy = CY(q), cz = CZ(q);
        const int xs = cx == 0 ? x : (cx > 0 ? s.xm : s.xp);
        bool w = false;
        if (WALLS) {
            if (cx > 0) w |= s.bxm;
            if (cx < 0) w |= s.bxp;
            if (cy > 0) w |= s.bym;
            if (cy < 0) w |= s.byp;
            if (cz > 0) w |= s.bzm;
            if (cz < 0) w |= s.bzp;
        }
        const long long a = w ? (long long)OPP(q) * g.ncell + s.own + x
                              : (long long)q * g.ncell + s.row[1 - cy][1 - cz] + xs;
        fc[q] = Storage<T>::load(grid + a);
    }
}

#define LBM_Q27_PROLOGUE                                    \
    const int x = blockIdx.x * blockDim.x + threadIdx.x;    \
    const int y = blockIdx.y * blockDim.y + threadIdx.y;    \
    const int z = blockIdx.z;                               \
    if (x >= g.nx || y >= g.ny) return;                     \
    const Site<true> s(x, y, z, 1, g);                      \
    const long long cell = s.own + x;

// f = feq(rho, u) (Eq. 14, shifted), written in the A/B layout.
template <typename T, typename In>
__global__ void k27_init(T *grid, const In *rho, const In *u, Geo g, Relax27<typename Storage<T>::R> p, int rho0_mode)
{
    using R = typename Storage<T>::R;
    LBM_Q27_PROLOGUE
    const R r = rho ? R(rho[cell]) : R(1);
    const R uv[3] = {R(u[cell]), R(u[g.ncell + cell]), R(u[2 * g.ncell + cell])};
    const R P = rho0_mode ? r : R(1);
    const R drho = r - R(1);
    const R uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
    const R base = drho - R(1.5) * P * uu;
    R fc[Q27];
    fc[0] = p.w[0] * base;
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        const int q = 2 * k + 1, cls = NORM2(q);
        const R cu = R(CX(q)) * uv[0] + R(CY(q)) * uv[1] + R(CZ(q)) * uv[2];
        const R sym = p.w[cls] * base + P * p.K[cls] * cu * cu;
        const R asym = R(0.5) * P * p.A[cls] * cu;
        fc[q] = sym + asym;
        fc[q + 1] = sym - asym;
    }
    put_canonical<T, true>(grid, s, x, g, fc);
}

template <typename T, typename Out>
__global__ void k27_moments(const T *__restrict__ grid, Out *rho, Out *u, Geo g, Relax27<typename Storage<T>::R> p,
                            int rho0_mode)
{
    using R = typename Storage<T>::R;
    LBM_Q27_PROLOGUE
    R fc[Q27];
    get_canonical<T, true>(grid, s, x, g, fc);
    R drho = fc[0], j[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int q = 1; q < Q27; ++q) {
        drho += fc[q];
        j[0] += R(CX(q)) * fc[q];
        j[1] += R(CY(q)) * fc[q];
        j[2] += R(CZ(q)) * fc[q];
    }
    const R inv = rho0_mode ? R(1) / (R(1) + drho) : R(1);
    if (rho) rho[cell] = Out(R(1) + drho);
    if (u)
        for (int i = 0; i < 3; ++i) u[i * g.ncell + cell] = Out((j[i] + p.half_a[i]) * inv);
}

template <typename T>
__global__ void k27_get(const T *__restrict__ grid, T *__restrict__ dst, Geo g)
{
    LBM_Q27_PROLOGUE
    typename Storage<T>::R fc[Q27];
    get_canonical<T, true>(grid, s, x, g, fc);
#pragma unroll
    for (int q = 0; q < Q27; ++q) Storage<T>::store(dst + (long long)q * g.ncell + cell, fc[q]);
}

template <typename T>
__global__ void k27_set(T *grid, const T *__restrict__ src, Geo g)
{
    LBM_Q27_PROLOGUE
    typename Storage<T>::R fc[Q27];
#pragma unroll
    for (int q = 0; q < Q27; ++q) fc[q] = Storage<T>::load(src + (long long)q * g.ncell + cell);
    put_canonical<T, true>(grid, s, x, g, fc);
}

}  // namespace q27

// ---------------------------------------------------------------- dispatch

template <typename F>
static cudaError_t q27_by_prec(int prec, F &&f)
{
    switch (prec) {
    case P_F64: return f(double());
    case P_F32: return f(float());
    case P_F16: return f(__half());
    case P_BF16: return f(__nv_bfloat16());
    }
    return cudaErrorInvalidValue;
}

static dim3 q27_block(const LaunchShape &s) { return dim3(s.bx, s.by, 1); }
static dim3 q27_grid(const Geo &g, const LaunchShape &s)
{
    return dim3((g.nx + s.bx - 1) / s.bx, (g.ny + s.by - 1) / s.by, g.nz);
}

cudaError_t launch_step27(int prec, const void *src, void *dst, const Geo &g, const CollBoth &c, LaunchShape s,
                          cudaStream_t stream)
{
    const bool walls = g.wall_x || g.wall_y || g.wall_z;
    return q27_by_prec(prec, [&](auto t) {
        using T = decltype(t);
        using R = typename Storage<T>::R;
        const q27::Relax27<R> p = q27::to_relax27<R>(c);
        const T *a = (const T *)src;
        T *b = (T *)dst;
        if constexpr (sizeof(T) == 2) {
            if (s.cells_x == 4 && g.nx % 4 == 0) {
                // four cells per thread; 128-thread blocks shaped as in the D3Q19 step
                const int nq = g.nx / 4;
                int bx = 128, idle = (nq + 127) / 128 * 128 - nq;
                for (int cw = 64; cw >= 32; cw /= 2) {
                    const int w = (nq + cw - 1) / cw * cw - nq;
                    if (w < idle) {
                        bx = cw;
                        idle = w;
                    }
                }
                const dim3 bl4(bx, 128 / bx, 1);
                // with walls, the interior rows run the periodic kernel (or with walls
                // on x the x-walls-only one) and the wall rows the walled one
                // (split_rows): walled channel 512x256x256, FP16, 0.68 -> 1.0 of the
                // copy bandwidth
                auto run = [&](auto rho0) {
                    constexpr bool RH = decltype(rho0)::value;
                    if (!walls) {
                        const dim3 gr4((g.nx + 4 * bx - 1) / (4 * bx), (g.ny + bl4.y - 1) / bl4.y, g.nz);
                        q27::k27_ab4<T, RH, false><<<gr4, bl4, 0, stream>>>(a, b, g, p, Rows{0, g.ny, 0});
                        return;
                    }
                    split_rows<true>(g, [&](int kind, Rows r, int nzr) {
                        const dim3 gr4((g.nx + 4 * bx - 1) / (4 * bx), (r.y1 - r.y0 + bl4.y - 1) / bl4.y, nzr);
                        if (kind == ROWS_WALLED)
                            q27::k27_ab4<T, RH, true, true><<<gr4, bl4, 0, stream>>>(a, b, g, p, r);
                        else if (kind == ROWS_XWALLS)
                            q27::k27_ab4<T, RH, true, true, true><<<gr4, bl4, 0, stream>>>(a, b, g, p, r);
                        else
                            q27::k27_ab4<T, RH, false, true><<<gr4, bl4, 0, stream>>>(a, b, g, p, r);
                    });
                };
                if (c.rho0_is_rho)
                    run(std::true_type{});
                else
                    run(std::false_type{});
                return cudaGetLastError();
            }
        }
        const dim3 gr = q27_grid(g, s), bl = q27_block(s);
        if (c.rho0_is_rho) {
            if (walls) q27::k27_ab1<T, true, true><<<gr, bl, 0, stream>>>(a, b, g, p);
            else q27::k27_ab1<T, true, false><<<gr, bl, 0, stream>>>(a, b, g, p);
        } else {
            if (walls) q27::k27_ab1<T, false, true><<<gr, bl, 0, stream>>>(a, b, g, p);
            else q27::k27_ab1<T, false, false><<<gr, bl, 0, stream>>>(a, b, g, p);
        }
        return cudaGetLastError();
    });
}

cudaError_t launch_init27(int prec, void *grid, const void *rho, const void *u, int dtype, const Geo &g,
                          const CollBoth &c, cudaStream_t stream)
{
    const LaunchShape s{128, 2, 1};
    return q27_by_prec(prec, [&](auto t) {
        using T = decltype(t);
        using R = typename Storage<T>::R;
        const q27::Relax27<R> p = q27::to_relax27<R>(c);
        if (dtype == 0)
            q27::k27_init<T, double><<<q27_grid(g, s), q27_block(s), 0, stream>>>((T *)grid, (const double *)rho,
                                                                                 (const double *)u, g, p,
                                                                                 c.rho0_is_rho);
        else
            q27::k27_init<T, float><<<q27_grid(g, s), q27_block(s), 0, stream>>>((T *)grid, (const float *)rho,
                                                                                (const float *)u, g, p,
                                                                                c.rho0_is_rho);
        return cudaGetLastError();
    });
}

cudaError_t launch_moments27(int prec, const void *grid, void *rho, void *u, int dtype, const Geo &g,
                             const CollBoth &c, cudaStream_t stream)
{
    const LaunchShape s{128, 2, 1};
    return q27_by_prec(prec, [&](auto t) {
        using T = decltype(t);
        using R = typename Storage<T>::R;
        const q27::Relax27<R> p = q27::to_relax27<R>(c);
        if (dtype == 0)
            q27::k27_moments<T, double><<<q27_grid(g, s), q27_block(s), 0, stream>>>(
                (const T *)grid, (double *)rho, (double *)u, g, p, c.rho0_is_rho);
        else
            q27::k27_moments<T, float><<<q27_grid(g, s), q27_block(s), 0, stream>>>(
                (const T *)grid, (float *)rho, (float *)u, g, p, c.rho0_is_rho);
        return cudaGetLastError();
    });
}

cudaError_t launch_get27(int prec, const void *grid, void *dst, const Geo &g, cudaStream_t stream)
{
    const LaunchShape s{128, 2, 1};
    return q27_by_prec(prec, [&](auto t) {
        using T = decltype(t);
        q27::k27_get<T><<<q27_grid(g, s), q27_block(s), 0, stream>>>((const T *)grid, (T *)dst, g);
        return cudaGetLastError();
    });
}

cudaError_t launch_set27(int prec, void *grid, const void *src, const Geo &g, cudaStream_t stream)
{
    const LaunchShape s{128, 2, 1};
    return q27_by_prec(prec, [&](auto t) {
        using T = decltype(t);
        q27::k27_set<T><<<q27_grid(g, s), q27_block(s), 0, stream>>>((T *)grid, (const T *)src, g);
        return cudaGetLastError();
    });
}

int velocity_set27(int *c, double *w, int *opp)
{
    for (int q = 0; q < q27::Q27; ++q) {
        if (c) {
            c[3 * q + 0] = q27::CX(q);
            c[3 * q + 1] = q27::CY(q);
            c[3 * q + 2] = q27::CZ(q);
        }
        if (w) w[q] = q27::WQ(q);
        if (opp) opp[q] = q27::OPP(q);
    }
    return q27::Q27;
}

}  // namespace lbm
