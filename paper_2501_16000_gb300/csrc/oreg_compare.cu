// olb_compare: the largest difference between the canonical populations of two
// lattices of the same size (any storage formats), reduced on the GPU, so that
// a reduced-precision state can be checked against an FP64 state over the
// whole of a large lattice without copying either to the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "oreg.h"
#include "oreg_aux.cuh"
#include "oreg_lattice.h"

using namespace oreg;

namespace {

constexpr int CMP_THREADS = 256;

struct Shift3 {
    double s[3];
};

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// out[0] = max |f_a - f_b|, out[1] = max |f_b| over every node and direction,
// as the bit patterns of non-negative doubles (whose order is that of the
// unsigned integers); a difference that is not finite counts as infinite.
template <int SA, int SB>
__global__ void __launch_bounds__(CMP_THREADS)
    k_compare(const typename Storage<SA>::T *a, StateGeom ga, Shift3 sa,
              const typename Storage<SB>::T *b, StateGeom gb, Shift3 sb,
              unsigned long long *out) {
    const long long N = (long long)ga.nx * ga.ny;
    double dmax = 0.0, rmax = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(n / ga.nx), x = (int)(n % ga.nx);
        double fa[9], fb[9];
        canon_node<SA>(a, x, y, ga, sa.s, fa);
        canon_node<SB>(b, x, y, gb, sb.s, fb);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double d = fabs(fa[i] - fb[i]);
            dmax = fmax(dmax, isfinite(d) ? d : INFINITY);
            rmax = fmax(rmax, isfinite(fb[i]) ? fabs(fb[i]) : INFINITY);
        }
    }
    dmax = warp_max(dmax);
    rmax = warp_max(rmax);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(dmax));
        atomicMax(&out[1], (unsigned long long)__double_as_longlong(rmax));
    }
}

template <int SA, int SB>
cudaError_t launch(const olb_lattice *A, const olb_lattice *B, unsigned long long *out,
                   int blocks) {
    Shift3 sa, sb;
    for (int c = 0; c < 3; ++c) {
        sa.s[c] = A->kd.shift[c];
        sb.s[c] = B->kd.shift[c];
    }
    k_compare<SA, SB><<<blocks, CMP_THREADS, 0, A->stream>>>(
        static_cast<const typename Storage<SA>::T *>(state_base(A)), geom(A), sa,
        static_cast<const typename Storage<SB>::T *>(state_base(B)), geom(B), sb, out);
    return cudaGetLastError();
}

template <int SA>
cudaError_t launch_b(const olb_lattice *A, const olb_lattice *B, unsigned long long *out,
                     int blocks) {
    switch (B->p.storage) {
        case OLB_F64: return launch<SA, ST_F64>(A, B, out, blocks);
        case OLB_F32: return launch<SA, ST_F32>(A, B, out, blocks);
        case OLB_F16_SHIFTED: return launch<SA, ST_F16>(A, B, out, blocks);
        default: return launch<SA, ST_BF16>(A, B, out, blocks);
    }
}

olb_status cmp_fail(olb_status st, const char *what, cudaError_t e = cudaSuccess) {
    char msg[256];
    if (e == cudaErrorMemoryAllocation) (void)cudaGetLastError();  // not sticky: clear it
    if (e != cudaSuccess) snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    else snprintf(msg, sizeof msg, "%s", what);
    set_last_error_message(msg);
    return st;
}

}  // namespace

extern "C" olb_status olb_compare(olb_lattice *a, olb_lattice *b, double *max_abs_diff,
                                  double *max_abs_ref) {
    if (!a || !b || !max_abs_diff) return cmp_fail(OLB_ERR_INVALID, "a, b and max_abs_diff must not be NULL");
    if (a->t < 0 || b->t < 0) return cmp_fail(OLB_ERR_STATE, "both lattices must be initialised");
    if (a->p.nx != b->p.nx || a->p.ny != b->p.ny)
        return cmp_fail(OLB_ERR_INVALID, "the lattices differ in size");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cmp_fail(OLB_ERR_CUDA, "waiting for the reference lattice", e);
    if (!a->d_cmp) {
        e = cudaMalloc(&a->d_cmp, 2 * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            a->d_cmp = nullptr;
            return cmp_fail(e == cudaErrorMemoryAllocation ? OLB_ERR_NOMEM : OLB_ERR_CUDA,
                            "allocating comparison scratch", e);
        }
    }
    e = cudaMemsetAsync(a->d_cmp, 0, 2 * sizeof(unsigned long long), a->stream);
    if (e != cudaSuccess) return cmp_fail(OLB_ERR_CUDA, "clearing comparison scratch", e);
    const long long N = (long long)a->p.nx * a->p.ny;
    const int blocks = (int)std::max<long long>(
        1, std::min<long long>((N + CMP_THREADS - 1) / CMP_THREADS, 8LL * a->num_sms));
    switch (a->p.storage) {
        case OLB_F64: e = launch_b<ST_F64>(a, b, a->d_cmp, blocks); break;
        case OLB_F32: e = launch_b<ST_F32>(a, b, a->d_cmp, blocks); break;
        case OLB_F16_SHIFTED: e = launch_b<ST_F16>(a, b, a->d_cmp, blocks); break;
        default: e = launch_b<ST_BF16>(a, b, a->d_cmp, blocks); break;
    }
    if (e != cudaSuccess) return cmp_fail(OLB_ERR_CUDA, "launching the comparison", e);
    unsigned long long h[2] = {0, 0};
    e = cudaMemcpyAsync(h, a->d_cmp, sizeof h, cudaMemcpyDeviceToHost, a->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(a->stream);
    if (e != cudaSuccess) return cmp_fail(OLB_ERR_CUDA, "reading the comparison", e);
    double d, r;
    static_assert(sizeof d == sizeof h[0], "double is 64-bit");
    memcpy(&d, &h[0], sizeof d);
    memcpy(&r, &h[1], sizeof r);
    *max_abs_diff = d;
    if (max_abs_ref) *max_abs_ref = r;
    return OLB_OK;
}
