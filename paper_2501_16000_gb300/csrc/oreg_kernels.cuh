// Stream-collide kernel templates (A-B pull, in-place AA) and their launcher,
// instantiated once per storage format (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "oreg_device.cuh"
#include "oreg_launch.h"

namespace oreg {

// Blocks of the largest size (256 threads) that the capped odd AA step must
// fit per SM, which caps its registers: 2 for the half formats (128
// registers, 16 warps resident; the issue-bound half formats need them, and
// the kernel would otherwise take ~140 registers), 3 for FP32 (85 registers,
// 24 warps for the HBM-bound kernel).  The periodic fixed-temperature kernels
// of these formats use the capped kernel; the wall and local-temperature
// variants need more registers and keep the compiler's own choice.
__host__ __device__ constexpr int step_min_blocks(int S) {
    return S == ST_F16 || S == ST_BF16 ? 2 : 3;
}
template <int S, int EQ, bool WALLS>
__host__ __device__ constexpr bool aa_odd_capped() {
    return !WALLS && EQ != EQ_GUIDED_LOCAL && (S == ST_F16 || S == ST_BF16 || S == ST_F32);
}

// ---------------------------------------------------------------------------
// Stream-collide, A-B layout.  A buffer holds post-collision populations at
// the node that produced them.  A warp gathers, for the 32*V nodes of a pass,
// f_i(x) = post_i(x - c_i) from src (the streaming of Eqs. 1/7 as a pull),
// which is the pre-collision state S_t(x); it collides and stores post(x) to
// dst at x.
// ---------------------------------------------------------------------------
template <int S, int I, bool AA_ODD>
__device__ __forceinline__ RawRow<S> fetch_plane(const typename Storage<S>::T *base, size_t plane,
                                                 int pitch, int y, int ny, int xb, int nx,
                                                 int sub, int W) {
    // A-B: population i at x comes from plane i at x - c_i.
    // AA odd step: it comes from plane opp(i) at x - c_i (written there by the
    // preceding even step).
    constexpr int P = AA_ODD ? opp_of(I) : I;
    const int ys = wrap_row(y - cy_of(I), ny);
    return fetch_row<S, cx_of(I), !AA_ODD>(base + P * plane + (size_t)ys * pitch, xb, nx, sub, W);
}

// Gathers the pre-collision populations of the warp pass's 32*V nodes: all
// nine row fetches are issued before any is decoded.
template <int S, bool AA_ODD>
__device__ __forceinline__ void pull_all(const typename Storage<S>::T *base, size_t plane,
                                         int pitch, int y, int ny, int xb, int nx, int sub, int W,
                                         typename Storage<S>::C f[9][Storage<S>::V]) {
    const RawRow<S> r0 = fetch_plane<S, 0, AA_ODD>(base, plane, pitch, y, ny, xb, nx, sub, W);
    const RawRow<S> r1 = fetch_plane<S, 1, AA_ODD>(base, plane, pitch, y, ny, xb, nx, sub, W);
    const RawRow<S> r2 = fetch_plane<S, 2, AA_ODD>(base, plane, pitch, y, ny, xb, nx, sub, W);
    const RawRow<S> r3 = fetch_plane<S, 3, AA_ODD>(base, plane, pitch, y, ny, xb, nx, sub, W);
    const RawRow<S> r4 = fetch_plane<S, 4, AA_ODD>(base, plane, pitch, y, ny, xb, nx, sub, W);
    const RawRow<S> r5 = fetch_plane<S, 5, AA_ODD>(base, plane, pitch, y, ny, xb, nx, sub, W);
    const RawRow<S> r6 = fetch_plane<S, 6, AA_ODD>(base, plane, pitch, y, ny, xb, nx, sub, W);
    const RawRow<S> r7 = fetch_plane<S, 7, AA_ODD>(base, plane, pitch, y, ny, xb, nx, sub, W);
    const RawRow<S> r8 = fetch_plane<S, 8, AA_ODD>(base, plane, pitch, y, ny, xb, nx, sub, W);
    shift_row<S, cx_of(0)>(r0, xb, nx, sub, W, f[0]);
    shift_row<S, cx_of(1)>(r1, xb, nx, sub, W, f[1]);
    shift_row<S, cx_of(2)>(r2, xb, nx, sub, W, f[2]);
    shift_row<S, cx_of(3)>(r3, xb, nx, sub, W, f[3]);
    shift_row<S, cx_of(4)>(r4, xb, nx, sub, W, f[4]);
    shift_row<S, cx_of(5)>(r5, xb, nx, sub, W, f[5]);
    shift_row<S, cx_of(6)>(r6, xb, nx, sub, W, f[6]);
    shift_row<S, cx_of(7)>(r7, xb, nx, sub, W, f[7]);
    shift_row<S, cx_of(8)>(r8, xb, nx, sub, W, f[8]);
}

// Row padding (positions nx .. pitch-1 of the last vector of a row) gets g = 0
// (the AA push may also copy finite node values there): never a non-finite.
template <int S>
__device__ __forceinline__ void zero_padding(typename Storage<S>::C f[9][Storage<S>::V], int xb,
                                             int nx) {
#pragma unroll
    for (int j = 0; j < Storage<S>::V; ++j)
        if (xb + j >= nx)
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i][j] = typename Storage<S>::C(0);
}

// Encodes the post-collision values to the storage format: round to nearest,
// or (half formats, sr) stochastically with counter-based bits per node,
// time step and direction.
// Half formats encode node pairs (x, x+1), x even, with one packed
// conversion; the stochastic draw of pair p of the lane (x = xb + 2p) and
// direction i is h + (9p + i) pair_step(h), h = node_seed(xb / V, y, t).
template <int S>
__device__ __forceinline__ void encode_vec(const typename Storage<S>::C f[9][Storage<S>::V],
                                           typename Storage<S>::T e[9][Storage<S>::V], int xb,
                                           int y, long long t, bool sr) {
    using ST = Storage<S>;
    using T = typename ST::T;
    if constexpr (S == ST_F16 || S == ST_BF16) {
        uint32_t w[9][ST::V / 2];
        if (sr) {
            const uint32_t h = node_seed(xb / ST::V, y, t), d = pair_step(h);
            uint32_t r = h;
#pragma unroll
            for (int j = 0; j < ST::V; j += 2) {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    w[i][j / 2] = ST::enc2_stochastic(f[i][j], f[i][j + 1], r);
                    r += d;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < ST::V; j += 2)
#pragma unroll
                for (int i = 0; i < 9; ++i) w[i][j / 2] = ST::enc2(f[i][j], f[i][j + 1]);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int j = 0; j < ST::V; j += 2) {
                const unsigned short lo = (unsigned short)(w[i][j / 2] & 0xFFFFu);
                const unsigned short hi = (unsigned short)(w[i][j / 2] >> 16);
                e[i][j] = *reinterpret_cast<const T *>(&lo);
                e[i][j + 1] = *reinterpret_cast<const T *>(&hi);
            }
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int j = 0; j < ST::V; ++j) e[i][j] = ST::enc_step(f[i][j]);
    }
}

// The collision constants broadcast to both lanes of a packed pair.
__device__ __forceinline__ CollConst<F2> broadcast(const CollConst<float> &k) {
    CollConst<F2> b;
    b.rho0 = F2(k.rho0);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        b.psi0[a] = F2(k.psi0[a]);
        b.psi0_lo[a] = F2(k.psi0_lo[a]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        b.w[c] = F2(k.w[c]);
        b.w_lo[c] = F2(k.w_lo[c]);
        b.shift[c] = F2(k.shift[c]);
        b.corr[c] = F2(k.corr[c]);
    }
    b.sum_corr = F2(k.sum_corr);
    b.sigma = F2(k.sigma);
    b.lam = F2(k.lam);
    b.inv_2th2 = F2(k.inv_2th2);
    b.theta = F2(k.theta);
    return b;
}

// Collides the V nodes of a lane.  The half formats (V = 8, FP32 compute,
// issue-bound) collide node pairs with packed f32x2 arithmetic; FP32 storage
// (HBM-bound) stays scalar, where packing measured no faster for A-B and
// slower for AA.
//
// FP32 with exact conserved sums forms them for node pairs with packed
// arithmetic (measured faster than per node in every layout; each lane
// rounds as the scalar operation, so the results are the same).
template <int S, int EQ, int COLL, bool EXACT>
__device__ __forceinline__ void collide_vec(typename Storage<S>::C f[9][Storage<S>::V],
                                            const CollConst<typename Storage<S>::C> &k) {
    using C = typename Storage<S>::C;
    if constexpr ((S == ST_F16 || S == ST_BF16) && !EXACT) {
        const CollConst<F2> k2 = broadcast(k);
#pragma unroll
        for (int j = 0; j < Storage<S>::V; j += 2) {
            F2 g[9], post[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = F2(f[i][j], f[i][j + 1]);
            collide<EQ, COLL, F2, false>(g, post, k2);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f[i][j] = post[i].lo();
                f[i][j + 1] = post[i].hi();
            }
        }
    } else if constexpr (S == ST_F32 && EXACT) {
        // the exact conserved sums of node pairs with packed arithmetic (the
        // split costs ~50 additions per node), the rest of the collision scalar
        CollConst<F2> k2;
        k2.sigma = F2(k.sigma);
        k2.sum_corr = F2(k.sum_corr);
#pragma unroll
        for (int j = 0; j < Storage<S>::V; j += 2) {
            F2 g2[9], m2[3];
#pragma unroll
            for (int i = 0; i < 9; ++i) g2[i] = F2(f[i][j], f[i][j + 1]);
            conserved<F2, true>(g2, k2, m2[0], m2[1], m2[2]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                C g[9], post[9];
                const C mom[3] = {h ? m2[0].hi() : m2[0].lo(), h ? m2[1].hi() : m2[1].lo(),
                                  h ? m2[2].hi() : m2[2].lo()};
#pragma unroll
                for (int i = 0; i < 9; ++i) g[i] = f[i][j + h];
                collide<EQ, COLL, C, EXACT, true>(g, post, k, mom);
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i][j + h] = post[i];
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < Storage<S>::V; ++j) {
            C g[9], post[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = f[i][j];
            collide<EQ, COLL, C, EXACT>(g, post, k);
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i][j] = post[i];
        }
    }
}

// Full-way bounce-back walls at columns 0 and nx - 1 (WALLS kernels only): a
// wall node does not collide; it returns every population along the link it
// arrived on, post_i(x) = f_opp(i)(x), with f the pre-collision state S_t.
// Called after collide_vec for lanes that hold a wall node, it reads the wall
// node's pre-collision values again from memory, which no thread has
// modified yet in any layout: A-B reads the unchanged source buffer; in the
// AA layout each location is read and written by its own node's update only,
// and this node's stores (including pushes by neighbouring lanes, whose
// values come from this lane through shuffles) come later.  MODE selects the
// addressing of f_k(x): A-B source plane k at x - c_k; AA even plane k at x;
// AA odd plane opp(k) at x - c_k.  The values are exact decodes of stored
// elements, so re-encoding them (also stochastically) returns the same bits.
template <int S, int MODE>
__device__ __forceinline__ void bounce_back_walls(const typename Storage<S>::T *base, size_t plane,
                                                  int pitch, int y, int ny, int xb, int nx,
                                                  typename Storage<S>::C f[9][Storage<S>::V]) {
    using ST = Storage<S>;
#pragma unroll
    for (int j = 0; j < ST::V; ++j) {
        const int x = xb + j;
        if (x == 0 || x == nx - 1) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int k = opp_of(i);
                size_t at;
                if (MODE == STATE_AA_EVEN) {
                    at = k * plane + (size_t)y * pitch + x;
                } else {
                    int xs = x - cx_of(k);
                    xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
                    const int p = MODE == STATE_AA_ODD ? opp_of(k) : k;
                    at = p * plane + (size_t)wrap_row(y - cy_of(k), ny) * pitch + xs;
                }
                f[i][j] = ST::dec_step(base[at]);
            }
        }
    }
}

// Whether the lane's nodes xb .. xb+V-1 include a wall column.
template <int S>
__device__ __forceinline__ bool lane_has_wall(int xb, int nx) {
    return xb < nx && (xb == 0 || xb + Storage<S>::V > nx - 1);
}

// The nodes of a lane in a warp pass.  A plane is pitch / V vectors per row,
// rows back to back (the pitch is nx rounded up to V), and a warp pass covers
// the 32 consecutive vectors v0 .. v0 + 31 of it in row-major order, so that
// its loads and stores are contiguous whatever the width; the lane holds
// vector v0 + lane: row y, nodes xb .. xb + V - 1.  Lanes past the last
// vector are idle (xb = nx) but still take part in the shuffles.  The
// shuffles run over the whole warp (W = 32, sub = lane); a lane whose
// neighbour lane holds another row (xb = 0, or its vector ends the row) takes
// the halo and wrap elements from memory instead.
template <int S>
__device__ __forceinline__ void lane_nodes(int v0, int lane, int nx, int ny, int pitch, int &y,
                                           int &xb) {
    constexpr unsigned V = Storage<S>::V;
    const unsigned vpr = (unsigned)pitch / V, v = (unsigned)(v0 + lane);
    const unsigned row = v / vpr;
    if (row >= (unsigned)ny) {
        y = ny - 1;
        xb = nx;
    } else {
        y = (int)row;
        xb = (int)((v - row * vpr) * V);
    }
}

// One warp pass of the A-B step: vectors v0 .. v0 + 31 of a lattice's planes.
template <int S, int EQ, int COLL, bool EXACT, bool WALLS>
__device__ __forceinline__ void item_ab(const typename Storage<S>::T *__restrict__ src,
                                        typename Storage<S>::T *__restrict__ dst, int nx, int ny,
                                        int pitch, size_t plane, int v0, int lane,
                                        const CollConst<typename Storage<S>::C> &k, long long t,
                                        bool sr) {
    using ST = Storage<S>;
    using C = typename ST::C;
    constexpr int V = ST::V;
    constexpr int W = 32;
    const int sub = lane;
    int y, xb;
    lane_nodes<S>(v0, lane, nx, ny, pitch, y, xb);

    C f[9][V];
    pull_all<S, false>(src, plane, pitch, y, ny, xb, nx, sub, W, f);

    collide_vec<S, EQ, COLL, EXACT>(f, k);
    if constexpr (WALLS) {
        if (lane_has_wall<S>(xb, nx))
            bounce_back_walls<S, STATE_AB>(src, plane, pitch, y, ny, xb, nx, f);
    }

    if (xb < nx) {
        if (xb + V > nx) zero_padding<S>(f, xb, nx);
        typename ST::T e[9][V];
        encode_vec<S>(f, e, xb, y, t, sr);
        typename ST::T *out = dst + (size_t)y * pitch + xb;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            Vec<S> v;
#pragma unroll
            for (int j = 0; j < V; ++j) v.e[j] = e[i][j];
            st_vec<S>(out + i * plane, v);
        }
    }
}

// One warp per warp pass; the grid covers them all.
#define OREG_AB_BODY                                                                        \
    const int pass = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);                   \
    if (pass >= passes) return; /* warp-uniform */                                          \
    item_ab<S, EQ, COLL, EXACT, WALLS>(src, dst, nx, ny, pitch, plane, pass << 5,             \
                                      threadIdx.x & 31, k, t, sr);

template <int S, int EQ, int COLL, bool EXACT, bool WALLS>
__global__ void __launch_bounds__(256) k_step_ab(const typename Storage<S>::T *__restrict__ src,
                                                 typename Storage<S>::T *__restrict__ dst, int nx,
                                                 int ny, int pitch, size_t plane, int passes,
                                                 const CollConst<typename Storage<S>::C> k,
                                                 long long t, bool sr) {
    OREG_AB_BODY
}

// The same A-B step for the issue-bound half formats, periodic and at a fixed
// temperature, with blocks of at most 128 threads: capped at 96 registers so
// that 5 blocks (20 warps) fit per SM instead of 4 (measured 2-4% faster; a
// small spill to L1 costs less than the lost warps).
template <int S, int EQ, bool WALLS>
__host__ __device__ constexpr bool ab_capped() {
    return !WALLS && EQ != EQ_GUIDED_LOCAL && (S == ST_F16 || S == ST_BF16);
}
constexpr int AB_CAPPED_MAX_THREADS = 128;
template <int S, int EQ, int COLL, bool EXACT, bool WALLS>
__global__ void __launch_bounds__(AB_CAPPED_MAX_THREADS, 5)
    k_step_ab_capped(const typename Storage<S>::T *__restrict__ src,
                     typename Storage<S>::T *__restrict__ dst, int nx, int ny, int pitch,
                     size_t plane, int passes, const CollConst<typename Storage<S>::C> k,
                     long long t, bool sr) {
    OREG_AB_BODY
}
#undef OREG_AB_BODY

// ---------------------------------------------------------------------------
// Stream-collide, in-place AA layout.
//   even step: read the node's own slots i, write post_i into slot opp(i);
//   odd step:  read slot opp(i) at x - c_i, write post_i into slot i at x + c_i.
// Every memory location is read and then written by the same node's update
// only, so the update is race-free in place.
// ---------------------------------------------------------------------------
template <int S, int EQ, int COLL, bool EXACT, bool WALLS>
__device__ __forceinline__ void item_aa_even(typename Storage<S>::T *A, int nx, int ny, int pitch,
                                             size_t plane, int v0, int lane,
                                             const CollConst<typename Storage<S>::C> &k,
                                             long long t, bool sr) {
    using ST = Storage<S>;
    using C = typename ST::C;
    constexpr int V = ST::V;
    int y, xb;
    lane_nodes<S>(v0, lane, nx, ny, pitch, y, xb);
    if (xb >= nx) return;  // no shuffles in the even step
    typename ST::T *row = A + (size_t)y * pitch + xb;
    C f[9][V];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        Vec<S> v = ld_vec<S>(row + i * plane);
#pragma unroll
        for (int j = 0; j < V; ++j) f[i][j] = ST::dec_step(v.e[j]);
    }
    collide_vec<S, EQ, COLL, EXACT>(f, k);
    if constexpr (WALLS) {
        if (lane_has_wall<S>(xb, nx))
            bounce_back_walls<S, STATE_AA_EVEN>(A, plane, pitch, y, ny, xb, nx, f);
    }
    if (xb + V > nx) zero_padding<S>(f, xb, nx);
    typename ST::T e[9][V];
    encode_vec<S>(f, e, xb, y, t, sr);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        Vec<S> v;
#pragma unroll
        for (int j = 0; j < V; ++j) v.e[j] = e[i][j];
        st_vec<S>(row + opp_of(i) * plane, v);
    }
}

template <int S, int EQ, int COLL, bool EXACT, bool WALLS>
__global__ void __launch_bounds__(256) k_step_aa_even(typename Storage<S>::T *A, int nx, int ny,
                                                      int pitch, size_t plane, int passes,
                                                      const CollConst<typename Storage<S>::C> k,
                                                      long long t, bool sr) {
    const int pass = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (pass >= passes) return;
    item_aa_even<S, EQ, COLL, EXACT, WALLS>(A, nx, ny, pitch, plane, pass << 5, threadIdx.x & 31,
                                           k, t, sr);
}

template <int S, int I>
__device__ __forceinline__ void push_plane(typename Storage<S>::T *A, size_t plane, int pitch,
                                           int y, int ny, int xb, int nx, int sub, int W,
                                           const typename Storage<S>::T p[Storage<S>::V]) {
    const int yd = wrap_row(y + cy_of(I), ny);
    store_row_shifted_raw<S, cx_of(I)>(A + I * plane + (size_t)yd * pitch, xb, nx, sub, W, p);
}

template <int S, int EQ, int COLL, bool EXACT, bool WALLS>
__device__ __forceinline__ void item_aa_odd(typename Storage<S>::T *A, int nx, int ny, int pitch,
                                            size_t plane, int v0, int lane,
                                            const CollConst<typename Storage<S>::C> &k,
                                            long long t, bool sr) {
    using ST = Storage<S>;
    using C = typename ST::C;
    constexpr int V = ST::V;
    constexpr int W = 32;
    const int sub = lane;
    int y, xb;
    lane_nodes<S>(v0, lane, nx, ny, pitch, y, xb);

    C f[9][V];
    pull_all<S, true>(A, plane, pitch, y, ny, xb, nx, sub, W, f);

    collide_vec<S, EQ, COLL, EXACT>(f, k);
    if constexpr (WALLS) {
        if (lane_has_wall<S>(xb, nx))
            bounce_back_walls<S, STATE_AA_ODD>(A, plane, pitch, y, ny, xb, nx, f);
    }
    if (xb < nx && xb + V > nx) zero_padding<S>(f, xb, nx);
    typename ST::T e[9][V];
    encode_vec<S>(f, e, xb, y, t, sr);

    push_plane<S, 0>(A, plane, pitch, y, ny, xb, nx, sub, W, e[0]);
    push_plane<S, 1>(A, plane, pitch, y, ny, xb, nx, sub, W, e[1]);
    push_plane<S, 2>(A, plane, pitch, y, ny, xb, nx, sub, W, e[2]);
    push_plane<S, 3>(A, plane, pitch, y, ny, xb, nx, sub, W, e[3]);
    push_plane<S, 4>(A, plane, pitch, y, ny, xb, nx, sub, W, e[4]);
    push_plane<S, 5>(A, plane, pitch, y, ny, xb, nx, sub, W, e[5]);
    push_plane<S, 6>(A, plane, pitch, y, ny, xb, nx, sub, W, e[6]);
    push_plane<S, 7>(A, plane, pitch, y, ny, xb, nx, sub, W, e[7]);
    push_plane<S, 8>(A, plane, pitch, y, ny, xb, nx, sub, W, e[8]);
}

#define OREG_AA_ODD_BODY                                                                    \
    const int pass = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);                   \
    if (pass >= passes) return;                                                             \
    item_aa_odd<S, EQ, COLL, EXACT, WALLS>(A, nx, ny, pitch, plane, pass << 5,                \
                                          threadIdx.x & 31, k, t, sr);

template <int S, int EQ, int COLL, bool EXACT, bool WALLS>
__global__ void __launch_bounds__(256) k_step_aa_odd(typename Storage<S>::T *A, int nx, int ny,
                                                     int pitch, size_t plane, int passes,
                                                     const CollConst<typename Storage<S>::C> k,
                                                     long long t, bool sr) {
    OREG_AA_ODD_BODY
}
template <int S, int EQ, int COLL, bool EXACT, bool WALLS>
__global__ void __launch_bounds__(256, step_min_blocks(S))
    k_step_aa_odd_capped(typename Storage<S>::T *A, int nx, int ny, int pitch, size_t plane,
                         int passes, const CollConst<typename Storage<S>::C> k, long long t,
                         bool sr) {
    OREG_AA_ODD_BODY
}
#undef OREG_AA_ODD_BODY

// ---------------------------------------------------------------------------
// Launcher
// ---------------------------------------------------------------------------
template <int S> struct StepLaunch {
    using ST = Storage<S>;
    using T = typename ST::T;
    using C = typename ST::C;

    template <int EQ, int COLL, bool EXACT, bool WALLS>
    static void step_eq(const StepArgs &a, dim3 grid, dim3 block) {
        const CollConst<C> &k = *static_cast<const CollConst<C> *>(a.kconst);
        const int passes = a.passes;
        if (a.layout == 0) {
            if constexpr (ab_capped<S, EQ, WALLS>()) {
                if (block.x <= (unsigned)AB_CAPPED_MAX_THREADS) {
                    k_step_ab_capped<S, EQ, COLL, EXACT, WALLS><<<grid, block, 0, a.stream>>>(
                        static_cast<const T *>(a.src), static_cast<T *>(a.dst), a.nx, a.ny,
                        a.pitch, a.plane, passes, k, a.t, a.sr != 0);
                    return;
                }
            }
            k_step_ab<S, EQ, COLL, EXACT, WALLS><<<grid, block, 0, a.stream>>>(
                static_cast<const T *>(a.src), static_cast<T *>(a.dst), a.nx, a.ny, a.pitch,
                a.plane, passes, k, a.t, a.sr != 0);
        } else if (a.parity == 0) {
            k_step_aa_even<S, EQ, COLL, EXACT, WALLS><<<grid, block, 0, a.stream>>>(
                static_cast<T *>(a.src), a.nx, a.ny, a.pitch, a.plane, passes, k, a.t,
                a.sr != 0);
        } else {
            if constexpr (aa_odd_capped<S, EQ, WALLS>()) {
                k_step_aa_odd_capped<S, EQ, COLL, EXACT, WALLS><<<grid, block, 0, a.stream>>>(
                    static_cast<T *>(a.src), a.nx, a.ny, a.pitch, a.plane, passes, k, a.t,
                    a.sr != 0);
            } else {
                k_step_aa_odd<S, EQ, COLL, EXACT, WALLS><<<grid, block, 0, a.stream>>>(
                    static_cast<T *>(a.src), a.nx, a.ny, a.pitch, a.plane, passes, k, a.t,
                    a.sr != 0);
            }
        }
    }

    template <bool EXACT, bool WALLS>
    static void step_comp(const StepArgs &a, dim3 grid, dim3 block) {
        if (a.eq == EQ_GUIDED) {
            if (a.coll == COLL_OREG) step_eq<EQ_GUIDED, COLL_OREG, EXACT, WALLS>(a, grid, block);
            else step_eq<EQ_GUIDED, COLL_BGK, EXACT, WALLS>(a, grid, block);
        } else if (a.eq == EQ_GUIDED_LOCAL) {
            if (a.coll == COLL_OREG) step_eq<EQ_GUIDED_LOCAL, COLL_OREG, EXACT, WALLS>(a, grid, block);
            else step_eq<EQ_GUIDED_LOCAL, COLL_BGK, EXACT, WALLS>(a, grid, block);
        } else {
            if (a.coll == COLL_OREG) step_eq<EQ_POLY2, COLL_OREG, EXACT, WALLS>(a, grid, block);
            else step_eq<EQ_POLY2, COLL_BGK, EXACT, WALLS>(a, grid, block);
        }
    }

    template <bool WALLS>
    static void step_walls(const StepArgs &a, dim3 grid, dim3 block) {
        // exact conserved sums exist for FP32 storage only
        if constexpr (S == ST_F32) {
            if (a.comp) {
                step_comp<true, WALLS>(a, grid, block);
                return;
            }
        }
        step_comp<false, WALLS>(a, grid, block);
    }

    static cudaError_t step(const StepArgs &a) {
        const int warps = a.warps_per_block;
        dim3 block(32 * warps);
        dim3 grid((unsigned)((a.passes + warps - 1) / warps));
        if (a.walls) step_walls<true>(a, grid, block);
        else step_walls<false>(a, grid, block);
        return cudaGetLastError();
    }
};

}  // namespace oreg
