// Auxiliary kernels of the OReg D2Q9 path: canonical-state access,
// initialisation, population readback/upload, moments and the FP64
// diagnostics reductions, with their launchers.
#pragma once

#include <cuda_runtime.h>

#include "oreg_device.cuh"
#include "oreg_kernels.cuh"
#include "oreg_launch.h"

namespace oreg {

// ---------------------------------------------------------------------------
// Canonical-state access (layout and parity aware), FP64.
//   A-B: the buffer holds the post-collision populations of the previous step
//        at the node where they were produced (the pull kernel gathers them
//        along -c_i before colliding), so S_t(x)_i = buf[i][x - c_i] + s_i.
//   AA, even t: S_t(x)_i = buf[i][x] + s_i.
//   AA, odd t:  S_t(x)_i = buf[opp(i)][x - c_i] + s_i.
// ---------------------------------------------------------------------------
template <int S>
__device__ __forceinline__ size_t canon_index(int i, int x, int y, const StateGeom &g) {
    if (g.mode == STATE_AA_EVEN) return i * g.plane + (size_t)y * g.pitch + x;
    int xs = x - cx_of(i), ys = y - cy_of(i);
    xs = xs < 0 ? xs + g.nx : (xs >= g.nx ? xs - g.nx : xs);
    ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
    const int p = g.mode == STATE_AA_ODD ? opp_of(i) : i;
    return p * g.plane + (size_t)ys * g.pitch + xs;
}

template <int S>
__device__ __forceinline__ void canon_node(const typename Storage<S>::T *base, int x, int y,
                                           const StateGeom &g, const double shift[3],
                                           double f[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        f[i] = (double)Storage<S>::dec(base[canon_index<S>(i, x, y, g)]) + shift[dcls(i)];
    }
}

// Equilibrium deviation f^eq_i - s_i in FP64 (used by the initialisers).
template <int EQ>
__device__ __forceinline__ void eq_dev_f64(double rho, double ux, double uy,
                                           const CollConst<double> &k, double geq[9]) {
    const double drho = rho - k.rho0;
    const double ux2 = ux * ux, uy2 = uy * uy;
    if constexpr (EQ == EQ_GUIDED) {
        const double dpx[3] = {-ux2, 0.5 * (ux + ux2), 0.5 * (ux2 - ux)};
        const double dpy[3] = {-uy2, 0.5 * (uy + uy2), 0.5 * (uy2 - uy)};
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int a = kidx(cx_of(i)), b = kidx(cy_of(i));
            const int pa = cx_of(i) != 0, pb = cy_of(i) != 0, ci = dcls(i);
            geq[i] = drho * (k.w[ci] + k.w_lo[ci]) +
                     rho * (dpx[a] * (k.psi0[pb] + dpy[b]) + k.psi0[pa] * dpy[b]) + k.corr[ci];
        }
    } else {
        const double u2 = ux2 + uy2;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double cu = cx_of(i) * ux + cy_of(i) * uy;
            const int ci = dcls(i);
            geq[i] = (k.w[ci] + k.w_lo[ci]) * (drho + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * u2)) +
                     k.corr[ci];
        }
    }
}

// S_0 = f^eq(rho(x), u(x)) written where the layout keeps S_0(x)_i.
template <int S, int EQ>
__global__ void k_init(typename Storage<S>::T *base, StateGeom g, InitSpec spec,
                       const CollConst<double> kd) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)g.nx * spec.rows) return;
    const int y = spec.y0 + (int)(n / g.nx), x = (int)(n % g.nx);
    double rho, ux, uy, exx = 0.0, eyy = 0.0, exy = 0.0;
    if (spec.mode == INIT_SHEAR) {
        // phase k.x / 2pi reduced exactly: (m x ny + n y nx) mod (nx ny)
        const long long N = (long long)g.nx * g.ny;
        long long num = ((long long)spec.m * x * g.ny + (long long)spec.n * y * g.nx) % N;
        if (num < 0) num += N;
        const double s = sinpi(2.0 * (double)num / (double)N);
        rho = spec.rho_a;
        ux = spec.ux_mean + spec.u0 * spec.ex * s;
        uy = spec.uy_mean + spec.u0 * spec.ey * s;
        if (spec.first_order) {
            // symmetric strain rate E = (grad u + grad u^T) / 2 of
            // u0 sin(k.x) e_perp: grad_b u_a = u0 cos(k.x) e_a k_b
            const double cph = spec.u0 * cospi(2.0 * (double)num / (double)N);
            exx = cph * spec.ex * spec.kx;
            eyy = cph * spec.ey * spec.ky;
            exy = 0.5 * cph * (spec.ex * spec.ky + spec.ey * spec.kx);
        }
    } else if (spec.mode == INIT_SHOCK) {
        rho = x < spec.x_split ? spec.rho_a : spec.rho_b;
        ux = 0.0;
        uy = 0.0;
    } else {
        rho = spec.rho[n];
        ux = spec.ux[n];
        uy = spec.uy[n];
    }
    double geq[9];
    eq_dev_f64<EQ>(rho, ux, uy, kd, geq);
    if (spec.mode == INIT_SHEAR && spec.first_order) {
        // Eq. 5: f_i^(1) = -(tau / theta) f_i^eq (C_ia C_ib - C_i^2 delta_ab / 2) E_ab,
        // C_i = c_i - u; the contraction with the symmetric E is
        // (Cx^2 - Cy^2)(Exx - Eyy)/2 + 2 Cx Cy Exy.
        const double a = -spec.tau / kd.theta;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double Cx = cx_of(i) - ux, Cy = cy_of(i) - uy;
            const double h = 0.5 * (Cx * Cx - Cy * Cy) * (exx - eyy) + 2.0 * Cx * Cy * exy;
            geq[i] += a * (geq[i] + kd.shift[dcls(i)]) * h;
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i)
        base[canon_index<S>(i, x, y, g)] = Storage<S>::enc((typename Storage<S>::C)geq[i]);
}

// Canonical populations of the window [x0, x0 + wx) x [y0, y0 + wy) into
// out[9][wy][wx] (FP64).
template <int S>
__global__ void k_get_canonical(const typename Storage<S>::T *base, StateGeom g, int x0, int y0,
                                int wx, int wy, const CollConst<double> kd, double *out) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long cnt = (long long)wx * wy;
    if (n >= cnt) return;
    const int y = y0 + (int)(n / wx), x = x0 + (int)(n % wx);
    double f[9];
    canon_node<S>(base, x, y, g, kd.shift, f);
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i * cnt + n] = f[i];
}

// Inverse: rows [y0, y0 + rows) of canonical FP64 populations into the state.
template <int S>
__global__ void k_set_canonical(typename Storage<S>::T *base, StateGeom g, int y0, int rows,
                                const CollConst<double> kd, const double *in) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long cnt = (long long)rows * g.nx;
    if (n >= cnt) return;
    const int y = y0 + (int)(n / g.nx), x = (int)(n % g.nx);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        base[canon_index<S>(i, x, y, g)] =
            Storage<S>::enc((typename Storage<S>::C)(in[i * cnt + n] - kd.shift[dcls(i)]));
    }
}

// Fields of rows [y0, y0 + rows): rho, u (Eq. 2a) and the local temperature.
template <int S>
__global__ void k_moments(const typename Storage<S>::T *base, StateGeom g, int y0, int rows,
                          const CollConst<double> kd, double *rho, double *ux, double *uy,
                          double *th) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long cnt = (long long)rows * g.nx;
    if (n >= cnt) return;
    const int y = y0 + (int)(n / g.nx), x = (int)(n % g.nx);
    double f[9];
    canon_node<S>(base, x, y, g, kd.shift, f);
    double r = 0, jx = 0, jy = 0, c2 = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        r += f[i];
        jx += cx_of(i) * f[i];
        jy += cy_of(i) * f[i];
        c2 += (cx_of(i) * cx_of(i) + cy_of(i) * cy_of(i)) * f[i];
    }
    const double vx = jx / r, vy = jy / r;
    rho[n] = r;
    if (ux) ux[n] = vx;
    if (uy) uy[n] = vy;
    if (th) th[n] = (c2 - r * (vx * vx + vy * vy)) / (2.0 * r);
}

// ---------------------------------------------------------------------------
// Diagnostics reductions (warp shuffles + shared memory), fixed grid, fixed
// order: deterministic.  Quantities: 0 sum of g over finite nodes, 1 momentum
// x, 2 momentum y, 3 non-finite node count, 4 and 5 mode projections
// sum u.e_perp sin(k.x) and sum u.e_perp cos(k.x).  The host adds the constant shifts back to the mass
// (N_finite sum_i s_i).
//
// Each thread accumulates in the storage's compute type C with error-free
// additions (hi + lo pairs, TwoSum), so FP32 formats keep FP64-grade sums
// while spending FP32 instructions; the per-thread pairs are combined in
// FP64.  sin(k.x) = sin(a) cos(b) + cos(a) sin(b),
// cos(k.x) = cos(a) cos(b) - sin(a) sin(b), a = 2 pi m x / nx,
// b = 2 pi n y / ny, from FP64 row/column tables built on the host.
// ---------------------------------------------------------------------------
constexpr int RED_Q = 6;
static_assert(RED_Q == RED_QUANTITIES, "reduction layout shared with the host");
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// (hi, lo) += x without rounding loss (lo collects the TwoSum remainders)
template <typename C>
__device__ __forceinline__ void pair_add(C &hi, C &lo, C x) {
    C s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
}

template <int S>
__global__ void __launch_bounds__(RED_THREADS) k_reduce(const typename Storage<S>::T *base,
                                                        StateGeom g, const CollConst<double> kd,
                                                        ModeSpec mode, double *partials) {
    using ST = Storage<S>;
    using C = typename ST::C;
    C hi[5] = {0, 0, 0, 0, 0}, lo[5] = {0, 0, 0, 0, 0};
    double nonfinite = 0.0;
    C sum_shift = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) sum_shift += (C)kd.shift[dcls(i)];
    const long long N = (long long)g.nx * g.ny;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // (x, y) of node n, advanced by the grid stride without a division per node
    int yn = (int)(n / g.nx), xn = (int)(n % g.nx);
    const int sy = (int)(stride / g.nx), sx = (int)(stride % g.nx);
    for (; n < N; n += stride) {
        const int y = yn, x = xn;
        xn += sx;
        yn += sy;
        if (xn >= g.nx) {
            xn -= g.nx;
            ++yn;
        }
        C v[9];
        bool finite = true;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            v[i] = ST::dec(base[canon_index<S>(i, x, y, g)]);
            finite = finite && isfinite(v[i]);
        }
        if (!finite) {
            nonfinite += 1.0;
            continue;
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            pair_add(hi[0], lo[0], v[i]);
            if (cx_of(i) != 0) pair_add(hi[1], lo[1], cx_of(i) > 0 ? v[i] : -v[i]);
            if (cy_of(i) != 0) pair_add(hi[2], lo[2], cy_of(i) > 0 ? v[i] : -v[i]);
        }
        if (mode.active) {
            C m = 0, jx = 0, jy = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                m += v[i];
                jx += C(cx_of(i)) * v[i];
                jy += C(cy_of(i)) * v[i];
            }
            const C rho = m + sum_shift;
            const C sa = (C)mode.tab[x], ca = (C)mode.tab[g.nx + x];
            const C sb = (C)mode.tab[2 * g.nx + y], cb = (C)mode.tab[2 * g.nx + g.ny + y];
            const C up = (jx * (C)mode.ex + jy * (C)mode.ey) / rho;
            pair_add(hi[3], lo[3], up * (sa * cb + ca * sb));
            pair_add(hi[4], lo[4], up * (ca * cb - sa * sb));
        }
    }
    double acc[RED_Q] = {(double)hi[0] + (double)lo[0], (double)hi[1] + (double)lo[1],
                         (double)hi[2] + (double)lo[2], nonfinite,
                         (double)hi[3] + (double)lo[3], (double)hi[4] + (double)lo[4]};
    __shared__ double sh[RED_THREADS / 32][RED_Q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < RED_Q; ++q) {
        const double val = warp_sum(acc[q]);
        if (lane == 0) sh[warp][q] = val;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < RED_Q; ++q) {
            double val = lane < RED_THREADS / 32 ? sh[lane][q] : 0.0;
            val = warp_sum(val);
            if (lane == 0) partials[(size_t)blockIdx.x * RED_Q + q] = val;
        }
    }
}

template <int S>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_final(const double *partials, int nblocks,
                                                              double *out) {
    double acc[RED_Q] = {};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < RED_Q; ++q) acc[q] += partials[(size_t)b * RED_Q + q];
    __shared__ double sh[RED_THREADS / 32][RED_Q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < RED_Q; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) sh[warp][q] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < RED_Q; ++q) {
            double v = lane < RED_THREADS / 32 ? sh[lane][q] : 0.0;
            v = warp_sum(v);
            if (lane == 0) out[q] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <int S> struct AuxLaunch {
    using ST = Storage<S>;
    using T = typename ST::T;
    using C = typename ST::C;

    static cudaError_t init(void *base, const StateGeom &g, const InitSpec &spec, int eq,
                            const CollConst<double> &kd, cudaStream_t s) {
        const long long N = (long long)g.nx * spec.rows;
        dim3 block(256), grid((unsigned)((N + 255) / 256));
        if (eq == EQ_GUIDED) k_init<S, EQ_GUIDED><<<grid, block, 0, s>>>(static_cast<T *>(base), g, spec, kd);
        else k_init<S, EQ_POLY2><<<grid, block, 0, s>>>(static_cast<T *>(base), g, spec, kd);
        return cudaGetLastError();
    }

    static cudaError_t get_canonical(const void *base, const StateGeom &g, int x0, int y0, int wx,
                                     int wy, const CollConst<double> &kd, double *out,
                                     cudaStream_t s) {
        const long long N = (long long)wx * wy;
        dim3 block(256), grid((unsigned)((N + 255) / 256));
        k_get_canonical<S><<<grid, block, 0, s>>>(static_cast<const T *>(base), g, x0, y0, wx, wy,
                                                  kd, out);
        return cudaGetLastError();
    }

    static cudaError_t set_canonical(void *base, const StateGeom &g, int y0, int rows,
                                     const CollConst<double> &kd, const double *in,
                                     cudaStream_t s) {
        const long long N = (long long)rows * g.nx;
        dim3 block(256), grid((unsigned)((N + 255) / 256));
        k_set_canonical<S><<<grid, block, 0, s>>>(static_cast<T *>(base), g, y0, rows, kd, in);
        return cudaGetLastError();
    }

    static cudaError_t moments(const void *base, const StateGeom &g, int y0, int rows,
                               const CollConst<double> &kd, double *rho, double *ux, double *uy,
                               double *th, cudaStream_t s) {
        const long long N = (long long)rows * g.nx;
        dim3 block(256), grid((unsigned)((N + 255) / 256));
        k_moments<S><<<grid, block, 0, s>>>(static_cast<const T *>(base), g, y0, rows, kd, rho,
                                            ux, uy, th);
        return cudaGetLastError();
    }

    static cudaError_t reduce(const void *base, const StateGeom &g, const CollConst<double> &kd,
                              const ModeSpec &mode, double *partials, int nblocks, double *out,
                              cudaStream_t s) {
        k_reduce<S><<<nblocks, RED_THREADS, 0, s>>>(static_cast<const T *>(base), g, kd, mode,
                                                     partials);
        k_reduce_final<S><<<1, RED_THREADS, 0, s>>>(partials, nblocks, out);
        return cudaGetLastError();
    }
};

}  // namespace oreg

#define OREG_DEFINE_LAUNCHERS(SUFFIX, S)                                                          \
    namespace oreg {                                                                              \
    cudaError_t step_##SUFFIX(const StepArgs &a) { return StepLaunch<S>::step(a); }               \
    cudaError_t init_##SUFFIX(void *b, const StateGeom &g, const InitSpec &sp, int eq,            \
                              const CollConst<double> &kd, cudaStream_t s) {                      \
        return AuxLaunch<S>::init(b, g, sp, eq, kd, s);                                              \
    }                                                                                             \
    cudaError_t get_canonical_##SUFFIX(const void *b, const StateGeom &g, int x0, int y0, int wx, \
                                       int wy, const CollConst<double> &kd, double *out,          \
                                       cudaStream_t s) {                                          \
        return AuxLaunch<S>::get_canonical(b, g, x0, y0, wx, wy, kd, out, s);                        \
    }                                                                                             \
    cudaError_t set_canonical_##SUFFIX(void *b, const StateGeom &g, int y0, int rows,             \
                                       const CollConst<double> &kd, const double *in,             \
                                       cudaStream_t s) {                                          \
        return AuxLaunch<S>::set_canonical(b, g, y0, rows, kd, in, s);                               \
    }                                                                                             \
    cudaError_t moments_##SUFFIX(const void *b, const StateGeom &g, int y0, int rows,             \
                                 const CollConst<double> &kd, double *r, double *ux, double *uy,  \
                                 double *th, cudaStream_t s) {                                    \
        return AuxLaunch<S>::moments(b, g, y0, rows, kd, r, ux, uy, th, s);                          \
    }                                                                                             \
    cudaError_t reduce_##SUFFIX(const void *b, const StateGeom &g, const CollConst<double> &kd,   \
                                const ModeSpec &m, double *partials, int nblocks, double *out,    \
                                cudaStream_t s) {                                                 \
        return AuxLaunch<S>::reduce(b, g, kd, m, partials, nblocks, out, s);                         \
    }                                                                                             \
    }
