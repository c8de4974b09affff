// Reverse-mode adjoint of the D3Q19 step (rho0 = 1).
//
// Forward map of one step: state(t+1) = S(C(state(t))), C the collision of
// Eq. 15 (or its TRT split) per cell, S the streaming permutation with
// half-way bounce-back.  The adjoint applies S^T (a gather from x + c_q, or
// from the opposite slot through a wall) and then C^T per cell.  With
// mu = S^T lambda(t+1), mu+/- the symmetric / antisymmetric parts over
// opposite pairs and nu = omega+ mu+ + omega- mu-, the transposed Jacobian of
// the collision is
//     lambda_p = mu_p - omega+ mu+_p - omega- mu-_p + sum_q nu_q dfeq_q/df_p,
//     dfeq_q/df_p = w_q + c_p . dfeq_q/du     (d rho/d f_p = 1, d u/d f_p = c_p),
// so lambda_p = mu_p - omega+ mu+_p - omega- mu-_p + A + c_p . G with
// A = sum_q w_q nu_q and G = sum_q nu_q dfeq_q/du.  For feq = D3Q19-S +
// kappa * Delta (see lbm_device.cuh),
//     sum_q nu_q dfeq^S_q/du = 3 B + 9 Cm u - 3 A u,
// B = sum_q w_q nu_q c_q, Cm = sum_q w_q nu_q c_q c_q^T, and the Delta part
// adds, per component i, nu_0 u_i / 3 - (u_i / 6)(sum of the face-pair sums
// on the two other axes) + (u_i / 12)(sum of nu over the edges normal to i).
// The step's derivatives with respect to omega+ and omega- are
//     dL/domega+ = -sum_q mu+_q (f_q - feq_q),
//     dL/domega- = -sum_q mu-_q (f_q - feq_q) - 1/2 sum_q mu_q F_q.
#include "lbm_device.cuh"
#include "lbm_launch.h"
#include "lbm_step.cuh"  // Planes, Site, gather1 (the A/B pull of the forward step)

namespace lbm {

static dim3 adj_block() { return dim3(128, 2, 1); }
static dim3 adj_grid(const Geo &g) { return dim3((g.nx + 127) / 128, (g.ny + 1) / 2, g.nz); }
int adjoint_blocks(const Geo &g)
{
    dim3 gr = adj_grid(g);
    return (int)(gr.x * gr.y * gr.z);
}

// G = sum_q nu_q dfeq_q/du and A = sum_q w_q nu_q at velocity u.
template <typename R>
__device__ __forceinline__ void contract_dfeq_du(const R nu[Q], const R u[3], R kappa, R G[3], R &A)
{
    R a = WQ<R>(0) * nu[0];
    R b[3] = {R(0), R(0), R(0)};
    R cxx = R(0), cyy = R(0), czz = R(0), cxy = R(0), cxz = R(0), cyz = R(0);
    R face[3] = {R(0), R(0), R(0)};  // nu summed over the two faces of each axis
    R edge[3] = {R(0), R(0), R(0)};  // nu summed over the four edges normal to each axis
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const R w = WQ<R>(q);
        const R wn = w * nu[q];
        a += wn;
        if (CX(q)) b[0] += R(CX(q)) * wn;
        if (CY(q)) b[1] += R(CY(q)) * wn;
        if (CZ(q)) b[2] += R(CZ(q)) * wn;
        if (CX(q)) cxx += wn;
        if (CY(q)) cyy += wn;
        if (CZ(q)) czz += wn;
        if (CX(q) * CY(q)) cxy += R(CX(q) * CY(q)) * wn;
        if (CX(q) * CZ(q)) cxz += R(CX(q) * CZ(q)) * wn;
        if (CY(q) * CZ(q)) cyz += R(CY(q) * CZ(q)) * wn;
        if (NORM2(q) == 1) {
            face[CX(q) ? 0 : (CY(q) ? 1 : 2)] += nu[q];
        } else {
            edge[CX(q) == 0 ? 0 : (CY(q) == 0 ? 1 : 2)] += nu[q];
        }
    }
    const R cu[3] = {cxx * u[0] + cxy * u[1] + cxz * u[2], cxy * u[0] + cyy * u[1] + cyz * u[2],
                     cxz * u[0] + cyz * u[1] + czz * u[2]};
    const R fs = face[0] + face[1] + face[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R gs = R(3) * b[i] + R(9) * cu[i] - R(3) * a * u[i];
        R gd = nu[0] * u[i] * (R(1) / R(3)) - u[i] * (fs - face[i]) * (R(1) / R(6)) + u[i] * edge[i] * (R(1) / R(12));
        G[i] = gs + kappa * gd;
    }
    A = a;
}

template <typename L>
__global__ void k_adjoint_seed(const void *grad_rho, const void *grad_u, int dtype, L *lam, Geo g)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long cell = ((long long)z * g.ny + y) * g.nx + x;
    double gu[3], gr = 0.0;
    for (int i = 0; i < 3; ++i)
        gu[i] = dtype == 0 ? ((const double *)grad_u)[i * g.ncell + cell] : ((const float *)grad_u)[i * g.ncell + cell];
    if (grad_rho) gr = dtype == 0 ? ((const double *)grad_rho)[cell] : ((const float *)grad_rho)[cell];
#pragma unroll
    for (int q = 0; q < Q; ++q)
        lam[(long long)q * g.ncell + cell] = L(CX(q) * gu[0] + CY(q) * gu[1] + CZ(q) * gu[2] + gr);
}

// Collision constants of the adjoint step: the forward step's folded
// constants (to recompute the collision) plus omega-, kappa and the raw force
// terms F_q = 3 w_q c_q . a of the pairs.
template <typename R>
struct AdjConst {
    Relax<R> r;
    R wm, kappa;
    R fraw[9];
};

template <typename R>
static inline AdjConst<R> to_adj(const CollBoth &c)
{
    AdjConst<R> a;
    a.r = to_relax<R>(c);
    a.wm = R(c.omega_m);
    a.kappa = R(c.kappa);
    for (int k = 0; k < 9; ++k) {
        const int q = 2 * k + 1;
        a.fraw[k] = R(3.0 * WQ<double>(q) * 2.0 *
                      (CX(q) * c.half_a[0] + CY(q) * c.half_a[1] + CZ(q) * c.half_a[2]));
    }
    return a;
}

template <typename R, int k>
__device__ __forceinline__ void adj_pair(const CellEq<R, false> &e, const R mu[Q], const R fraw[9], R &cgp, R &cgm,
                                         R &cf)
{
    constexpr int q = 2 * k + 1;
    R nsym, nasym;
    e.template neq<k>(nsym, nasym);
    const R S = mu[q] + mu[q + 1], D = mu[q] - mu[q + 1];
    cgp += S * nsym;
    cgm += D * nasym;
    cf += D * fraw[k];
}

// Double-float numbers: an unevaluated sum hi + lo of two floats.  Sums of
// FP32 terms built with error-free transformations (TwoSum) keep about 48
// bits, as many as FP64 sums of the same FP32 terms would, and run on the FP32
// pipe.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const float s = a.hi + b.hi;
    const float bv = s - a.hi;
    float e = (a.hi - (s - bv)) + (b.hi - bv);
    e += a.lo + b.lo;
    const float hi = s + e;
    return DF{hi, e - (hi - s)};
}

__device__ __forceinline__ DF df_warp_sum(DF a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DF b{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
        a = df_add(a, b);
    }
    return a;
}

// The adjoint of one cell: from the forward populations f of the state at t
// (rho0 = 1) and mu = S^T lambda(t+1), the cell's lambda(t) (out) and its
// terms of dL/domega+ (gp) and dL/domega- (gm).
template <typename R>
__device__ __forceinline__ void adjoint_cell(const R f[Q], const R mu[Q], const AdjConst<R> &p, R out[Q], R &gp,
                                             R &gm)
{
    const CellEq<R, false> e(f, p.r);
    // omega gradients of this cell:
    //   sum_q mu+_q (f - feq)_q = mu0 (f0 - feq0) + 1/2 sum_k S_k (s - 2 sym)_k
    //   sum_q mu-_q (f - feq)_q = 1/2 sum_k D_k (d - 2 asym)_k
    R cgp = R(0), cgm = R(0), cf_ = R(0);
    adj_pair<R, 0>(e, mu, p.fraw, cgp, cgm, cf_);
    adj_pair<R, 1>(e, mu, p.fraw, cgp, cgm, cf_);
    adj_pair<R, 2>(e, mu, p.fraw, cgp, cgm, cf_);
    adj_pair<R, 3>(e, mu, p.fraw, cgp, cgm, cf_);
    adj_pair<R, 4>(e, mu, p.fraw, cgp, cgm, cf_);
    adj_pair<R, 5>(e, mu, p.fraw, cgp, cgm, cf_);
    adj_pair<R, 6>(e, mu, p.fraw, cgp, cgm, cf_);
    adj_pair<R, 7>(e, mu, p.fraw, cgp, cgm, cf_);
    adj_pair<R, 8>(e, mu, p.fraw, cgp, cgm, cf_);
    gp = -(mu[0] * (f[0] - e.eq0) + R(0.5) * cgp);
    gm = R(-0.5) * (cgm + cf_);
    // lambda_p = mu_p - omega+ mu+_p - omega- mu-_p + A + c_p . G
    R Ssum_f = R(0), Ssum_e = R(0);
    R face[3] = {R(0), R(0), R(0)}, edge[3] = {R(0), R(0), R(0)};
    R Bd[3] = {R(0), R(0), R(0)};
    R cxx = R(0), cyy = R(0), czz = R(0), cxy = R(0), cxz = R(0), cyz = R(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int q = 2 * k + 1;
        const R S = mu[q] + mu[q + 1], D = mu[q] - mu[q + 1];
        const R w = WQ<R>(q);
        if (NORM2(q) == 1) {
            Ssum_f += S;
            face[CX(q) ? 0 : (CY(q) ? 1 : 2)] += S;
        } else {
            Ssum_e += S;
            edge[CX(q) == 0 ? 0 : (CY(q) == 0 ? 1 : 2)] += S;
        }
        const R wD = w * D, wS = w * S;
        if (CX(q)) Bd[0] += R(CX(q)) * wD;
        if (CY(q)) Bd[1] += R(CY(q)) * wD;
        if (CZ(q)) Bd[2] += R(CZ(q)) * wD;
        if (CX(q)) cxx += wS;
        if (CY(q)) cyy += wS;
        if (CZ(q)) czz += wS;
        if (CX(q) * CY(q)) cxy += R(CX(q) * CY(q)) * wS;
        if (CX(q) * CZ(q)) cxz += R(CX(q) * CZ(q)) * wS;
        if (CY(q) * CZ(q)) cyz += R(CY(q) * CZ(q)) * wS;
    }
    const R wp = p.r.wp;
    const R A = wp * (WQ<R>(0) * mu[0] + WQ<R>(1) * Ssum_f + WQ<R>(7) * Ssum_e);
    const R *u = e.u;
    const R cu3[3] = {cxx * u[0] + cxy * u[1] + cxz * u[2], cxy * u[0] + cyy * u[1] + cyz * u[2],
                      cxz * u[0] + cyz * u[1] + czz * u[2]};
    const R fs = face[0] + face[1] + face[2];
    R G[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const R gs = R(3) * p.wm * Bd[i] + R(9) * wp * cu3[i] - R(3) * A * u[i];
        const R gd = wp * (mu[0] * (R(1) / R(3)) - (fs - face[i]) * (R(1) / R(6)) + edge[i] * (R(1) / R(12)));
        G[i] = gs + p.kappa * gd * u[i];
    }
    out[0] = (R(1) - wp) * mu[0] + A;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int q = 2 * k + 1;
        const R S = mu[q] + mu[q + 1], D = mu[q] - mu[q + 1];
        const R cg = R(CX(q)) * G[0] + R(CY(q)) * G[1] + R(CZ(q)) * G[2];
        const R t = A - p.r.hp * S;
        const R hd = p.r.hm * D;
        out[q] = mu[q] + t - hd + cg;
        out[q + 1] = mu[q + 1] + t + hd - cg;
    }
}

// Fixed-order sum of the per-block partials of k_adjoint_step into
// grad_omega: FP64 partials (FP64 storage) in FP64, the double-float partials
// of the FP32 arithmetic in double-float, the result added to grad_omega in
// FP64.  The order is that of ADJ_SUM_VIRT virtual threads: virtual thread v
// adds partials v, v + ADJ_SUM_VIRT, v + 2 ADJ_SUM_VIRT, ... in turn; the 32
// virtual threads of each virtual warp are reduced by one shuffle tree and the
// 32 virtual-warp sums by one more.  A block of NT threads (a multiple of 32,
// blockDim.x a multiple of 32) plays ADJ_SUM_VIRT / NT virtual threads per
// thread with the same lanes, so the result is bitwise the same for every NT:
// the sum can run as its own one-block kernel (NT = 1024) or in one block of
// the next adjoint step (NT = 256, see lbm_adjoint_step with deferred sums).
constexpr int ADJ_SUM_VIRT = 1024;

struct AccD {
    double a0, a1;
};
struct AccF {
    DF a0, a1;
};
__device__ __forceinline__ void acc_add(AccD &a, const double2 &v)
{
    a.a0 += v.x;
    a.a1 += v.y;
}
__device__ __forceinline__ void acc_add(AccF &a, const float4 &v)
{
    a.a0 = df_add(a.a0, DF{v.x, v.y});
    a.a1 = df_add(a.a1, DF{v.z, v.w});
}
__device__ __forceinline__ AccD acc_warp_sum(AccD a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a.a0 += __shfl_down_sync(0xffffffffu, a.a0, o);
        a.a1 += __shfl_down_sync(0xffffffffu, a.a1, o);
    }
    return a;
}
__device__ __forceinline__ AccF acc_warp_sum(AccF a) { return AccF{df_warp_sum(a.a0), df_warp_sum(a.a1)}; }
__device__ __forceinline__ void acc_store(double *g, const AccD &a)
{
    g[0] += a.a0;
    g[1] += a.a1;
}
__device__ __forceinline__ void acc_store(double *g, const AccF &a)
{
    g[0] += (double)a.a0.hi + (double)a.a0.lo;
    g[1] += (double)a.a1.hi + (double)a.a1.lo;
}

// U terms of each virtual thread are loaded together (their order of addition
// does not change).  sh: ADJ_SUM_VIRT / 32 accumulators of shared memory.
template <int NT, int U, typename P, typename A>
__device__ __forceinline__ void sum_partials(const P *partial, long long nblocks, double *grad_omega, A *sh)
{
    constexpr int V = ADJ_SUM_VIRT / NT;
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    A acc[V];
#pragma unroll
    for (int k = 0; k < V; ++k) acc[k] = A{};
    for (long long j = 0; j < nblocks; j += (long long)U * ADJ_SUM_VIRT) {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const long long b0 = j + t + k * NT;
            P v[U];
#pragma unroll
            for (int i = 0; i < U; ++i) {
                const long long b = b0 + (long long)i * ADJ_SUM_VIRT;
                if (b < nblocks) v[i] = partial[b];
            }
#pragma unroll
            for (int i = 0; i < U; ++i)
                if (b0 + (long long)i * ADJ_SUM_VIRT < nblocks) acc_add(acc[k], v[i]);
        }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) acc[k] = acc_warp_sum(acc[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < V; ++k) sh[warp + k * (NT / 32)] = acc[k];
    }
    __syncthreads();
    if (warp == 0) {
        const A a = acc_warp_sum(sh[lane]);
        if (lane == 0) acc_store(grad_omega, a);
    }
}

// Addressing as in the forward step kernels: plane base pointers from the
// kernel parameters, nine wrapped row offsets per thread (Site), and no
// bounce-back logic when the lattice is periodic (WALLS = false).
// prev_partial (may be NULL): the partials of the previous adjoint step, whose
// sum the first block adds to prev_grad after its own cells (deferred sums).
template <typename T, typename L, bool WALLS>
__global__ void __launch_bounds__(256, sizeof(typename Storage<T>::R) == 8 ? 2 : 4)
    k_adjoint_step(Planes<T> state, Planes<L> lam_next, Planes<L> lam, double *partial, Geo g,
                   AdjConst<typename Storage<T>::R> p, const double *prev_partial, long long prev_nblocks,
                   double *prev_grad)
{
    using R = typename Storage<T>::R;
    __shared__ typename Storage<T>::R shp[256], shm[256];  // compute precision
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    R gp_cell = R(0), gm_cell = R(0);  // this cell's terms of dL/domega+ and dL/domega-
    if (x < g.nx && y < g.ny) {
        const Site<WALLS> st(x, y, z, 1, g);
        const int self = st.own + x;
        // forward populations of the cell at time t (rho0 = 1), and S^T: the
        // value that left x along c_q arrived at x + c_q (or, through a wall,
        // at the opposite slot of x).  All 38 loads are issued first.
        R f[Q], mu[Q];
        gather1<false>(state, st, f);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int cx = CX(q);
            const int xt = cx == 0 ? x : (cx > 0 ? st.xp : st.xm);
            bool w = st.template wall_yz<1>(q);
            if (WALLS) {
                if (cx > 0) w |= st.bxp;
                if (cx < 0) w |= st.bxm;
            }
            const L *a = w ? lam_next.p[OPP(q)] + self : lam_next.p[q] + st.template row_along<1>(q) + xt;
            mu[q] = R(*a);
        }
        R out[Q];
        adjoint_cell(f, mu, p, out, gp_cell, gm_cell);
#pragma unroll
        for (int q = 0; q < Q; ++q) lam.p[q][self] = L(out[q]);
    }
    // Block partial: the per-cell terms are staged in shared memory (in the
    // compute precision) and one warp sums them in a fixed order: in FP64 for
    // FP64 storage, in double-float (see below) for the FP32 arithmetic.
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    shp[tid] = gp_cell;
    shm[tid] = gm_cell;
    __syncthreads();
    if (tid < 32) {
        const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        if constexpr (sizeof(R) == 8) {
            double a0 = 0.0, a1 = 0.0;
            for (int i = tid; i < nthreads; i += 32) {
                a0 += (double)shp[i];
                a1 += (double)shm[i];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a0 += __shfl_down_sync(0xffffffffu, a0, o);
                a1 += __shfl_down_sync(0xffffffffu, a1, o);
            }
            if (tid == 0) reinterpret_cast<double2 *>(partial)[b] = make_double2(a0, a1);
        } else {
            DF a0{0.f, 0.f}, a1{0.f, 0.f};
            for (int i = tid; i < nthreads; i += 32) {
                two_sum_acc(a0.hi, a0.lo, (float)shp[i]);
                two_sum_acc(a1.hi, a1.lo, (float)shm[i]);
            }
            a0 = df_warp_sum(a0);
            a1 = df_warp_sum(a1);
            if (tid == 0) reinterpret_cast<float4 *>(partial)[b] = make_float4(a0.hi, a0.lo, a1.hi, a1.lo);
        }
    }
    if (prev_partial && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
        // the previous step has completed (stream order), its partials are visible
        if constexpr (sizeof(R) == 8) {
            __shared__ AccD sh[ADJ_SUM_VIRT / 32];
            sum_partials<256, 2>(reinterpret_cast<const double2 *>(prev_partial), prev_nblocks, prev_grad, sh);
        } else {
            __shared__ AccF sh[ADJ_SUM_VIRT / 32];
            sum_partials<256, 2>(reinterpret_cast<const float4 *>(prev_partial), prev_nblocks, prev_grad, sh);
        }
    }
    // the sum of the partials (launched as a programmatic dependent) may start
    // once every block has got here; it waits for this grid's memory itself
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The sum of the per-block partials of one adjoint step as a kernel of its
// own (one block of ADJ_SUM_VIRT threads, each thread's eight loads in flight
// together): launched as a programmatic dependent of the step, or by
// lbm_adjoint_flush.  Summing the 8192 partials of the 128^3 adjoint workload
// in FP64 on the one SM took 11 us, an eighth of the step, because this GPU's
// FP64 pipe is narrow; the double-float sums of the FP32 arithmetic run on the
// FP32 pipe.
template <typename P, typename A>
__global__ void __launch_bounds__(ADJ_SUM_VIRT) k_adjoint_final(const P *partial, long long nblocks,
                                                                double *grad_omega)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");  // k_adjoint_step has finished, its partials visible
    __shared__ A sh[ADJ_SUM_VIRT / 32];
    sum_partials<ADJ_SUM_VIRT, 8>(partial, nblocks, grad_omega, sh);
}

template <typename In, typename L, typename R>
__global__ void k_adjoint_init_velocity(const In *u0, const L *lam0, In *grad_u0, Geo g, R kappa)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long cell = ((long long)z * g.ny + y) * g.nx + x;
    R u[3] = {R(u0[cell]), R(u0[g.ncell + cell]), R(u0[2 * g.ncell + cell])};
    R nu[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) nu[q] = R(lam0[(long long)q * g.ncell + cell]);
    R G[3], A;
    contract_dfeq_du(nu, u, kappa, G, A);
    for (int i = 0; i < 3; ++i) grad_u0[i * g.ncell + cell] = In(G[i]);
}

// ---------------------------------------------------------------- dispatch

cudaError_t launch_adjoint_seed(int prec, const void *grad_rho, const void *grad_u, int dtype, void *lambda,
                                const Geo &g, cudaStream_t s)
{
    if (prec == P_F64)
        k_adjoint_seed<double><<<adj_grid(g), adj_block(), 0, s>>>(grad_rho, grad_u, dtype, (double *)lambda, g);
    else
        k_adjoint_seed<float><<<adj_grid(g), adj_block(), 0, s>>>(grad_rho, grad_u, dtype, (float *)lambda, g);
    return cudaGetLastError();
}

// One adjoint step.  partial: this step's block partials.  defer: leave them
// for the next step's first block (prev_partial / prev_grad of that launch) or
// for launch_adjoint_flush instead of summing them at once.
template <typename T, typename L>
static cudaError_t adj_step_t(const void *state, const void *lam_next, void *lam, double *grad_omega, double *partial,
                              const double *prev_partial, double *prev_grad, bool defer, const Geo &g,
                              const CollBoth &cb, cudaStream_t s)
{
    using R = typename Storage<T>::R;
    AdjConst<R> p = to_adj<R>(cb);
    const Planes<T> S = planes_of<T>(const_cast<void *>(state), g.ncell);
    const Planes<L> Ln = planes_of<L>(const_cast<void *>(lam_next), g.ncell);
    const Planes<L> Lo = planes_of<L>(lam, g.ncell);
    const long long nb = adjoint_blocks(g);
    if (g.wall_x || g.wall_y || g.wall_z)
        k_adjoint_step<T, L, true><<<adj_grid(g), adj_block(), 0, s>>>(S, Ln, Lo, partial, g, p, prev_partial, nb,
                                                                      prev_grad);
    else
        k_adjoint_step<T, L, false><<<adj_grid(g), adj_block(), 0, s>>>(S, Ln, Lo, partial, g, p, prev_partial, nb,
                                                                       prev_grad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || defer) return e;
    // The final sum is a programmatic dependent launch: it is scheduled while
    // the step kernel's last blocks run (griddepcontrol.launch_dependents) and
    // waits inside for the step's completion (griddepcontrol.wait), which hides
    // the launch gap between the two.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, 1, 1);
    cfg.blockDim = dim3(ADJ_SUM_VIRT, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (sizeof(R) == 8)
        e = cudaLaunchKernelEx(&cfg, k_adjoint_final<double2, AccD>, reinterpret_cast<const double2 *>(partial), nb,
                               grad_omega);
    else
        e = cudaLaunchKernelEx(&cfg, k_adjoint_final<float4, AccF>, reinterpret_cast<const float4 *>(partial), nb,
                               grad_omega);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(int prec, const void *state, const void *lam_next, void *lam, double *grad_omega,
                                double *partial, const double *prev_partial, double *prev_grad, bool defer,
                                const Geo &g, const CollBoth &c, cudaStream_t s)
{
#define LBM_ADJ_ARGS state, lam_next, lam, grad_omega, partial, prev_partial, prev_grad, defer, g, c, s
    switch (prec) {
    case P_F64: return adj_step_t<double, double>(LBM_ADJ_ARGS);
    case P_F32: return adj_step_t<float, float>(LBM_ADJ_ARGS);
    case P_F16: return adj_step_t<__half, float>(LBM_ADJ_ARGS);
    case P_BF16: return adj_step_t<__nv_bfloat16, float>(LBM_ADJ_ARGS);
    }
#undef LBM_ADJ_ARGS
    return cudaErrorInvalidValue;
}

// Sums the deferred partials of an adjoint step into grad_omega.
cudaError_t launch_adjoint_flush(int prec, const double *partial, double *grad_omega, const Geo &g, cudaStream_t s)
{
    const long long nb = adjoint_blocks(g);
    if (prec == P_F64)
        k_adjoint_final<double2, AccD><<<1, ADJ_SUM_VIRT, 0, s>>>(reinterpret_cast<const double2 *>(partial), nb,
                                                                 grad_omega);
    else
        k_adjoint_final<float4, AccF><<<1, ADJ_SUM_VIRT, 0, s>>>(reinterpret_cast<const float4 *>(partial), nb,
                                                                grad_omega);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_init_velocity(int prec, const void *rho, const void *u0, int dtype, const void *lam0,
                                         void *grad_u0, const Geo &g, const CollBoth &c, cudaStream_t s)
{
    (void)rho;  // with rho0 = 1, dfeq/du does not depend on rho
    if (prec == P_F64) {
        if (dtype == 0)
            k_adjoint_init_velocity<double, double, double><<<adj_grid(g), adj_block(), 0, s>>>(
                (const double *)u0, (const double *)lam0, (double *)grad_u0, g, c.kappa);
        else
            k_adjoint_init_velocity<float, double, double><<<adj_grid(g), adj_block(), 0, s>>>(
                (const float *)u0, (const double *)lam0, (float *)grad_u0, g, c.kappa);
    } else {
        if (dtype == 0)
            k_adjoint_init_velocity<double, float, float><<<adj_grid(g), adj_block(), 0, s>>>(
                (const double *)u0, (const float *)lam0, (double *)grad_u0, g, (float)c.kappa);
        else
            k_adjoint_init_velocity<float, float, float><<<adj_grid(g), adj_block(), 0, s>>>(
                (const float *)u0, (const float *)lam0, (float *)grad_u0, g, (float)c.kappa);
    }
    return cudaGetLastError();
}

}  // namespace lbm
