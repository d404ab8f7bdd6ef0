// Kernel templates of the OReg D2Q9 path and their launchers, instantiated once
// per storage format (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "oreg_device.cuh"
#include "oreg_launch.h"

namespace oreg {

// ---------------------------------------------------------------------------
// Stream-collide, A-B layout.  A buffer holds post-collision populations at
// the node that produced them.  A warp gathers, for 32*V nodes of one row,
// f_i(x) = post_i(x - c_i) from src (the streaming of Eqs. 1/7 as a pull),
// which is the pre-collision state S_t(x); it collides and stores post(x) to
// dst at x.
// ---------------------------------------------------------------------------
template <int S, int I, bool AA_ODD>
__device__ __forceinline__ void pull_plane(const typename Storage<S>::T *base, size_t plane,
                                           int pitch, int y, int ny, int xb, int nx, int lane,
                                           typename Storage<S>::C out[Storage<S>::V]) {
    // A-B: population i at x comes from plane i at x - c_i.
    // AA odd step: it comes from plane opp(i) at x - c_i (written there by the
    // preceding even step).
    constexpr int P = AA_ODD ? opp_of(I) : I;
    const int ys = wrap_row(y - cy_of(I), ny);
    load_row_shifted<S, cx_of(I), !AA_ODD>(base + P * plane + (size_t)ys * pitch, xb, nx, lane,
                                            out);
}

// Row padding (positions nx .. pitch-1 of the last vector of a row) is kept
// at g = 0 so that it never holds values that are not finite.
template <int S>
__device__ __forceinline__ void zero_padding(typename Storage<S>::C f[9][Storage<S>::V], int xb,
                                             int nx) {
#pragma unroll
    for (int j = 0; j < Storage<S>::V; ++j)
        if (xb + j >= nx)
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i][j] = typename Storage<S>::C(0);
}

template <int S, int EQ, int COLL, bool COMP>
__device__ __forceinline__ void collide_vec(typename Storage<S>::C f[9][Storage<S>::V],
                                            const CollConst<typename Storage<S>::C> &k) {
    using C = typename Storage<S>::C;
#pragma unroll
    for (int j = 0; j < Storage<S>::V; ++j) {
        C g[9], post[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = f[i][j];
        collide<EQ, COLL, C, COMP>(g, post, k);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i][j] = post[i];
    }
}

template <int S, int EQ, int COLL, bool COMP>
__global__ void __launch_bounds__(256) k_step_ab(const typename Storage<S>::T *__restrict__ src,
                                                 typename Storage<S>::T *__restrict__ dst, int nx,
                                                 int ny, int pitch, size_t plane, int segs,
                                                 const CollConst<typename Storage<S>::C> k) {
    using ST = Storage<S>;
    using C = typename ST::C;
    constexpr int V = ST::V;
    const int lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= (long long)ny * segs) return;  // warp-uniform
    const int y = (int)(item / segs), seg = (int)(item % segs);
    const int xb = seg * 32 * V + lane * V;

    C f[9][V];
    pull_plane<S, 0, false>(src, plane, pitch, y, ny, xb, nx, lane, f[0]);
    pull_plane<S, 1, false>(src, plane, pitch, y, ny, xb, nx, lane, f[1]);
    pull_plane<S, 2, false>(src, plane, pitch, y, ny, xb, nx, lane, f[2]);
    pull_plane<S, 3, false>(src, plane, pitch, y, ny, xb, nx, lane, f[3]);
    pull_plane<S, 4, false>(src, plane, pitch, y, ny, xb, nx, lane, f[4]);
    pull_plane<S, 5, false>(src, plane, pitch, y, ny, xb, nx, lane, f[5]);
    pull_plane<S, 6, false>(src, plane, pitch, y, ny, xb, nx, lane, f[6]);
    pull_plane<S, 7, false>(src, plane, pitch, y, ny, xb, nx, lane, f[7]);
    pull_plane<S, 8, false>(src, plane, pitch, y, ny, xb, nx, lane, f[8]);

    collide_vec<S, EQ, COLL, COMP>(f, k);

    if (xb < nx) {
        if (xb + V > nx) zero_padding<S>(f, xb, nx);
        typename ST::T *out = dst + (size_t)y * pitch + xb;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            Vec<S> v;
#pragma unroll
            for (int j = 0; j < V; ++j) v.e[j] = ST::enc(f[i][j]);
            st_vec<S>(out + i * plane, v);
        }
    }
}

// ---------------------------------------------------------------------------
// Stream-collide, in-place AA layout.
//   even step: read the node's own slots i, write post_i into slot opp(i);
//   odd step:  read slot opp(i) at x - c_i, write post_i into slot i at x + c_i.
// Every memory location is read and then written by the same node's update
// only, so the update is race-free in place.
// ---------------------------------------------------------------------------
template <int S, int EQ, int COLL, bool COMP>
__global__ void __launch_bounds__(256) k_step_aa_even(typename Storage<S>::T *A, int nx, int ny,
                                                      int pitch, size_t plane, int segs,
                                                      const CollConst<typename Storage<S>::C> k) {
    using ST = Storage<S>;
    using C = typename ST::C;
    constexpr int V = ST::V;
    const int lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= (long long)ny * segs) return;
    const int y = (int)(item / segs), seg = (int)(item % segs);
    const int xb = seg * 32 * V + lane * V;
    if (xb >= nx) return;  // no shuffles in this kernel
    typename ST::T *row = A + (size_t)y * pitch + xb;
    C f[9][V];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        Vec<S> v = ld_vec<S>(row + i * plane);
#pragma unroll
        for (int j = 0; j < V; ++j) f[i][j] = ST::dec(v.e[j]);
    }
    collide_vec<S, EQ, COLL, COMP>(f, k);
    if (xb + V > nx) zero_padding<S>(f, xb, nx);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        Vec<S> v;
#pragma unroll
        for (int j = 0; j < V; ++j) v.e[j] = ST::enc(f[i][j]);
        st_vec<S>(row + opp_of(i) * plane, v);
    }
}

template <int S, int I>
__device__ __forceinline__ void push_plane(typename Storage<S>::T *A, size_t plane, int pitch,
                                           int y, int ny, int xb, int nx, int lane,
                                           const typename Storage<S>::C p[Storage<S>::V]) {
    const int yd = wrap_row(y + cy_of(I), ny);
    store_row_shifted<S, cx_of(I)>(A + I * plane + (size_t)yd * pitch, xb, nx, lane, p);
}

template <int S, int EQ, int COLL, bool COMP>
__global__ void __launch_bounds__(256) k_step_aa_odd(typename Storage<S>::T *A, int nx, int ny,
                                                     int pitch, size_t plane, int segs,
                                                     const CollConst<typename Storage<S>::C> k) {
    using ST = Storage<S>;
    using C = typename ST::C;
    constexpr int V = ST::V;
    const int lane = threadIdx.x & 31;
    const long long item = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= (long long)ny * segs) return;
    const int y = (int)(item / segs), seg = (int)(item % segs);
    const int xb = seg * 32 * V + lane * V;

    C f[9][V];
    pull_plane<S, 0, true>(A, plane, pitch, y, ny, xb, nx, lane, f[0]);
    pull_plane<S, 1, true>(A, plane, pitch, y, ny, xb, nx, lane, f[1]);
    pull_plane<S, 2, true>(A, plane, pitch, y, ny, xb, nx, lane, f[2]);
    pull_plane<S, 3, true>(A, plane, pitch, y, ny, xb, nx, lane, f[3]);
    pull_plane<S, 4, true>(A, plane, pitch, y, ny, xb, nx, lane, f[4]);
    pull_plane<S, 5, true>(A, plane, pitch, y, ny, xb, nx, lane, f[5]);
    pull_plane<S, 6, true>(A, plane, pitch, y, ny, xb, nx, lane, f[6]);
    pull_plane<S, 7, true>(A, plane, pitch, y, ny, xb, nx, lane, f[7]);
    pull_plane<S, 8, true>(A, plane, pitch, y, ny, xb, nx, lane, f[8]);

    collide_vec<S, EQ, COLL, COMP>(f, k);
    if (xb < nx && xb + V > nx) zero_padding<S>(f, xb, nx);

    push_plane<S, 0>(A, plane, pitch, y, ny, xb, nx, lane, f[0]);
    push_plane<S, 1>(A, plane, pitch, y, ny, xb, nx, lane, f[1]);
    push_plane<S, 2>(A, plane, pitch, y, ny, xb, nx, lane, f[2]);
    push_plane<S, 3>(A, plane, pitch, y, ny, xb, nx, lane, f[3]);
    push_plane<S, 4>(A, plane, pitch, y, ny, xb, nx, lane, f[4]);
    push_plane<S, 5>(A, plane, pitch, y, ny, xb, nx, lane, f[5]);
    push_plane<S, 6>(A, plane, pitch, y, ny, xb, nx, lane, f[6]);
    push_plane<S, 7>(A, plane, pitch, y, ny, xb, nx, lane, f[7]);
    push_plane<S, 8>(A, plane, pitch, y, ny, xb, nx, lane, f[8]);
}

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
                                           const StateGeom &g, const double shift[9],
                                           double f[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        f[i] = (double)Storage<S>::dec(base[canon_index<S>(i, x, y, g)]) + shift[i];
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
            geq[i] = drho * (k.w[i] + k.w_lo[i]) +
                     rho * (dpx[a] * (k.psi0[b] + dpy[b]) + k.psi0[a] * dpy[b]) + k.corr[i];
        }
    } else {
        const double u2 = ux2 + uy2;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double cu = cx_of(i) * ux + cy_of(i) * uy;
            geq[i] = (k.w[i] + k.w_lo[i]) * (drho + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * u2)) +
                     k.corr[i];
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
    double rho, ux, uy;
    if (spec.mode == INIT_SHEAR) {
        // phase k.x / 2pi reduced exactly: (m x ny + n y nx) mod (nx ny)
        const long long N = (long long)g.nx * g.ny;
        long long num = ((long long)spec.m * x * g.ny + (long long)spec.n * y * g.nx) % N;
        if (num < 0) num += N;
        const double s = sinpi(2.0 * (double)num / (double)N);
        rho = spec.rho_a;
        ux = spec.u0 * spec.ex * s;
        uy = spec.u0 * spec.ey * s;
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
            Storage<S>::enc((typename Storage<S>::C)(in[i * cnt + n] - kd.shift[i]));
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
// FP64 reductions (warp shuffles + shared memory), fixed grid, fixed order:
// deterministic.  Quantities: 0 mass, 1 momentum x, 2 momentum y,
// 3 non-finite node count, 4 mode projection sum u.e_perp sin(k.x).
// ---------------------------------------------------------------------------
constexpr int RED_Q = 5;
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int S>
__global__ void __launch_bounds__(RED_THREADS) k_reduce(const typename Storage<S>::T *base,
                                                        StateGeom g, const CollConst<double> kd,
                                                        ModeSpec mode, double *partials) {
    double acc[RED_Q] = {0, 0, 0, 0, 0};
    const long long N = (long long)g.nx * g.ny;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(n / g.nx), x = (int)(n % g.nx);
        double f[9];
        canon_node<S>(base, x, y, g, kd.shift, f);
        double r = 0, jx = 0, jy = 0;
        bool finite = true;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            finite = finite && isfinite(f[i]);
            r += f[i];
            jx += cx_of(i) * f[i];
            jy += cy_of(i) * f[i];
        }
        if (!finite) {
            acc[3] += 1.0;
            continue;
        }
        acc[0] += r;
        acc[1] += jx;
        acc[2] += jy;
        if (mode.active) {
            const long long M = N;
            long long num = ((long long)mode.m * x * g.ny + (long long)mode.n * y * g.nx) % M;
            if (num < 0) num += M;
            const double s = sinpi(2.0 * (double)num / (double)M);
            acc[4] += (jx * mode.ex + jy * mode.ey) / r * s;
        }
    }
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
            if (lane == 0) partials[(size_t)blockIdx.x * RED_Q + q] = v;
        }
    }
}

template <int S>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_final(const double *partials, int nblocks,
                                                              double *out) {
    double acc[RED_Q] = {0, 0, 0, 0, 0};
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
template <int S> struct Launch {
    using ST = Storage<S>;
    using T = typename ST::T;
    using C = typename ST::C;

    template <int EQ, int COLL, bool COMP>
    static void step_eq(const StepArgs &a, dim3 grid, dim3 block) {
        const CollConst<C> &k = *static_cast<const CollConst<C> *>(a.kconst);
        const int segs = a.segs;
        if (a.layout == 0) {
            k_step_ab<S, EQ, COLL, COMP><<<grid, block, 0, a.stream>>>(
                static_cast<const T *>(a.src), static_cast<T *>(a.dst), a.nx, a.ny, a.pitch,
                a.plane, segs, k);
        } else if (a.parity == 0) {
            k_step_aa_even<S, EQ, COLL, COMP><<<grid, block, 0, a.stream>>>(
                static_cast<T *>(a.src), a.nx, a.ny, a.pitch, a.plane, segs, k);
        } else {
            k_step_aa_odd<S, EQ, COLL, COMP><<<grid, block, 0, a.stream>>>(
                static_cast<T *>(a.src), a.nx, a.ny, a.pitch, a.plane, segs, k);
        }
    }

    template <bool COMP>
    static void step_comp(const StepArgs &a, dim3 grid, dim3 block) {
        if (a.eq == EQ_GUIDED) {
            if (a.coll == COLL_OREG) step_eq<EQ_GUIDED, COLL_OREG, COMP>(a, grid, block);
            else step_eq<EQ_GUIDED, COLL_BGK, COMP>(a, grid, block);
        } else {
            if (a.coll == COLL_OREG) step_eq<EQ_POLY2, COLL_OREG, COMP>(a, grid, block);
            else step_eq<EQ_POLY2, COLL_BGK, COMP>(a, grid, block);
        }
    }

    static cudaError_t step(const StepArgs &a) {
        const int warps = a.warps_per_block;
        const long long items = (long long)a.ny * a.segs;
        dim3 block(32 * warps);
        dim3 grid((unsigned)((items + warps - 1) / warps));
        if (a.comp && S == ST_F32) step_comp<true>(a, grid, block);
        else step_comp<false>(a, grid, block);
        return cudaGetLastError();
    }

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
    cudaError_t step_##SUFFIX(const StepArgs &a) { return Launch<S>::step(a); }                   \
    cudaError_t init_##SUFFIX(void *b, const StateGeom &g, const InitSpec &sp, int eq,            \
                              const CollConst<double> &kd, cudaStream_t s) {                      \
        return Launch<S>::init(b, g, sp, eq, kd, s);                                              \
    }                                                                                             \
    cudaError_t get_canonical_##SUFFIX(const void *b, const StateGeom &g, int x0, int y0, int wx, \
                                       int wy, const CollConst<double> &kd, double *out,          \
                                       cudaStream_t s) {                                          \
        return Launch<S>::get_canonical(b, g, x0, y0, wx, wy, kd, out, s);                        \
    }                                                                                             \
    cudaError_t set_canonical_##SUFFIX(void *b, const StateGeom &g, int y0, int rows,             \
                                       const CollConst<double> &kd, const double *in,             \
                                       cudaStream_t s) {                                          \
        return Launch<S>::set_canonical(b, g, y0, rows, kd, in, s);                               \
    }                                                                                             \
    cudaError_t moments_##SUFFIX(const void *b, const StateGeom &g, int y0, int rows,             \
                                 const CollConst<double> &kd, double *r, double *ux, double *uy,  \
                                 double *th, cudaStream_t s) {                                    \
        return Launch<S>::moments(b, g, y0, rows, kd, r, ux, uy, th, s);                          \
    }                                                                                             \
    cudaError_t reduce_##SUFFIX(const void *b, const StateGeom &g, const CollConst<double> &kd,   \
                                const ModeSpec &m, double *partials, int nblocks, double *out,    \
                                cudaStream_t s) {                                                 \
        return Launch<S>::reduce(b, g, kd, m, partials, nblocks, out, s);                         \
    }                                                                                             \
    }
