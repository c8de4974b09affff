// Fused stream + collide time step (Eq. 15; D3Q19-S / D3Q19-I equilibria;
// SRT / TRT; periodic or half-way bounce-back; Buick-Greated force).
//
// One thread updates one cell: it gathers the 19 populations that stream into
// the cell, collides them in registers (FP32, or FP64 for FP64 storage), and
// stores the 19 post-collision values.  Structure-of-arrays storage gives
// coalesced accesses along x for every population; the +-x populations are
// read one element off alignment, which L1/L2 absorb without extra DRAM
// traffic.  The algorithmic traffic is 19 loads + 19 stores per cell.
#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace lbm {

// A/B pull step: gather from src (layout AB), write dst in layout AB.
template <typename T>
__global__ void __launch_bounds__(256) k_step_ab(const T *__restrict__ src, T *__restrict__ dst, Geo g,
                                                 Coll<typename Storage<T>::R> p)
{
    using R = typename Storage<T>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    Cell c(x, y, z, g);
    R f[Q];
    gather<AB>(src, c, g.ncell, f);
    collide(f, p);
    scatter<D_AB_NEXT>(dst, c, g.ncell, f);
}

// AA in-place steps.  Even: own cell only (read q, write qbar).  Odd: read
// qbar at x - c_q, write q at x + c_q (bounce-back through walls stays in the
// own cell).  Every location is read and written by exactly one thread.
template <typename T, int ODD>
__global__ void __launch_bounds__(256) k_step_aa(T *grid, Geo g, Coll<typename Storage<T>::R> p)
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
        collide(f, p);
        scatter<D_AA_ODD>(grid, c, g.ncell, f);
    } else {
        gather<AA_EVEN>(grid, c, g.ncell, f);
        collide(f, p);
        scatter<D_AA_EVEN>(grid, c, g.ncell, f);
    }
}

template <typename T>
static cudaError_t step_t(int kind, const void *src, void *dst, const Geo &g, const CollBoth &cb, LaunchShape s,
                          cudaStream_t stream)
{
    using R = typename Storage<T>::R;
    Coll<R> p = to_coll<R>(cb);
    dim3 block(s.bx, s.by, 1);
    dim3 grid((g.nx + s.bx - 1) / s.bx, (g.ny + s.by - 1) / s.by, g.nz);
    if (kind == 0)
        k_step_ab<T><<<grid, block, 0, stream>>>((const T *)src, (T *)dst, g, p);
    else if (kind == 1)
        k_step_aa<T, 0><<<grid, block, 0, stream>>>((T *)dst, g, p);
    else
        k_step_aa<T, 1><<<grid, block, 0, stream>>>((T *)dst, g, p);
    return cudaGetLastError();
}

cudaError_t launch_step(int prec, int kind, const void *src, void *dst, const Geo &g, const CollBoth &c,
                        LaunchShape s, cudaStream_t stream)
{
    switch (prec) {
    case P_F64: return step_t<double>(kind, src, dst, g, c, s, stream);
    case P_F32: return step_t<float>(kind, src, dst, g, c, s, stream);
    case P_F16: return step_t<__half>(kind, src, dst, g, c, s, stream);
    case P_BF16: return step_t<__nv_bfloat16>(kind, src, dst, g, c, s, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
