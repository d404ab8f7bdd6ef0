// Device-side building blocks of the OReg D2Q9 stream-collide path (sm_103a).
//
//   * D2Q9 velocity set and opposite-direction table (Fig. 1a).
//   * Storage codecs: every format holds shifted populations g_i = f_i - s_i.
//   * The per-node collision: moments (Eq. 2a), guided (Eq. 11) or polynomial
//     (Eq. 15) equilibrium, the OReg projection (Eq. 6) and the update of
//     Eq. 7, or lattice BGK (Eq. 1), all written in deviation variables so
//     that no O(1) quantity is formed and then cancelled in low precision.
//   * Warp-level shifted row loads (pull streaming) and stores (push
//     streaming of the in-place AA layout) on 16-byte vectors.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace oreg {

// ---------------------------------------------------------------------------
// D2Q9 velocity set, order (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx_of(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
// Component index of a velocity component: 0 -> 0, +1 -> 1, -1 -> 2.
__host__ __device__ constexpr int kidx(int c) { return c == 0 ? 0 : (c > 0 ? 1 : 2); }
// Symmetry class of a direction: 0 rest, 1 axis, 2 diagonal (the rest
// weights, shifts and their corrections depend on the class only).
__host__ __device__ constexpr int dcls(int i) {
    return (cx_of(i) != 0 ? 1 : 0) + (cy_of(i) != 0 ? 1 : 0);
}

static_assert(opp_of(1) == 3 && opp_of(2) == 4 && opp_of(3) == 1 && opp_of(4) == 2, "opp");
static_assert(opp_of(5) == 7 && opp_of(6) == 8 && opp_of(7) == 5 && opp_of(8) == 6, "opp");

// Equilibrium kinds of the kernels: guided at the lattice's fixed theta,
// polynomial, and guided at each node's own temperature (local theta).
enum { EQ_GUIDED = 0, EQ_POLY2 = 1, EQ_GUIDED_LOCAL = 2 };
enum { COLL_OREG = 0, COLL_BGK = 1 };
enum { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3, ST_F32_C64 = 4 };

// ---------------------------------------------------------------------------
// Storage traits: T = stored element, C = compute type, V = elements per 16 B.
// ---------------------------------------------------------------------------
template <int S> struct Storage;
//
// dec/enc map stored elements to and from g = f - s (used by the auxiliary
// kernels with the FP64 constants).  The stream-collide kernels use
// dec_step/enc_step (and the packed enc2/enc2_stochastic of the half
// formats), which work in step units: g * STEP_SCALE.  The collision is
// homogeneous of degree one in (f, rho) (f^eq is linear in rho and f^OReg
// scales as f^eq S / rho), so the step kernels run it unchanged in units
// scaled by a power of two, with rho0, the shifts and their corrections
// scaled alike on the host; scaling by a power of two is exact, so this
// only removes two multiplications per element.
template <> struct Storage<ST_F64> {
    using T = double; using C = double; static constexpr int V = 2;
    static constexpr double STEP_SCALE = 1.0;
    __device__ static C dec(T v) { return v; }
    __device__ static T enc(C v) { return v; }
    __device__ static C dec_step(T v) { return v; }
    __device__ static T enc_step(C v) { return v; }
};
template <> struct Storage<ST_F32> {
    using T = float; using C = float; static constexpr int V = 4;
    static constexpr double STEP_SCALE = 1.0;
    __device__ static C dec(T v) { return v; }
    __device__ static T enc(C v) { return v; }
    __device__ static C dec_step(T v) { return v; }
    __device__ static T enc_step(C v) { return v; }
};
// FP32 storage with the collision in FP64 (option OLB_OPT_F64_COLLISION): the
// stored elements and shifts are those of ST_F32, so a state written by either
// kernel is read by the other; the only FP32 rounding left in a step is the
// store of the post-collision values.
template <> struct Storage<ST_F32_C64> {
    using T = float; using C = double; static constexpr int V = 4;
    static constexpr double STEP_SCALE = 1.0;
    __device__ static C dec(T v) { return v; }
    __device__ static T enc(C v) { return __double2float_rn(v); }
    __device__ static C dec_step(T v) { return v; }
    __device__ static T enc_step(C v) { return __double2float_rn(v); }
};
// Half formats also offer stochastic rounding: the bits of v below the
// format's last mantissa bit (13 for f16, 16 for bf16) get uniform random
// bits added before truncation, so v rounds away from zero with probability
// equal to its distance from the truncated value.
// f16 stores g * 2^8: the shifted populations are small (|g| ~ 1e-5 .. 1e-1
// in the benchmarks), and the scale keeps them above the f16 subnormal
// range (2^-14), where the format has fixed absolute resolution 2^-24.
// Scaling by a power of two is exact.  |g| must stay below 65504 / 2^8 = 255.
//
// Pairs of adjacent elements are encoded with one packed conversion:
// enc2 (round to nearest even) and enc2_stochastic, the sm_100-family
// stochastic-rounding conversion cvt.rs.{f16x2,bf16x2}.f32, which adds the
// low 13 (f16) or all 16 (bf16) bits of each 16-bit half of r to the
// discarded mantissa bits of the matching input (low half -> lo, high half
// -> hi) and truncates.  The result packs lo in the low and hi in the high
// 16 bits, the order in which the two elements sit in memory.
template <> struct Storage<ST_F16> {
    using T = __half; using C = float; static constexpr int V = 8;
    static constexpr float SCALE = 256.0f, INV_SCALE = 1.0f / 256.0f;
    static constexpr double STEP_SCALE = 256.0;  // step units are the stored units
    __device__ static C dec(T v) { return __half2float(v) * INV_SCALE; }
    __device__ static T enc(C v) { return __float2half_rn(v * SCALE); }
    __device__ static C dec_step(T v) { return __half2float(v); }
    __device__ static T enc_step(C v) { return __float2half_rn(v); }
    __device__ static uint32_t enc2(C lo, C hi) {
        const __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    __device__ static uint32_t enc2_stochastic(C lo, C hi, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
        return d;
    }
};
template <> struct Storage<ST_BF16> {
    using T = __nv_bfloat16; using C = float; static constexpr int V = 8;
    static constexpr double STEP_SCALE = 1.0;
    __device__ static C dec(T v) { return __bfloat162float(v); }
    __device__ static T enc(C v) { return __float2bfloat16_rn(v); }
    __device__ static C dec_step(T v) { return __bfloat162float(v); }
    __device__ static T enc_step(C v) { return __float2bfloat16_rn(v); }
    __device__ static uint32_t enc2(C lo, C hi) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    __device__ static uint32_t enc2_stochastic(C lo, C hi, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
        return d;
    }
};

// Counter-based random bits for stochastic rounding: one hash per group of V
// consecutive nodes (x0 = a multiple of V, the nodes of one lane) and time
// step (the 32-bit finalizer of MurmurHash3 of (x0/V, y, t)), then the words
// of its node pairs (x, x+1), x = x0 + 2p, and directions i as one arithmetic
// progression r = h + (9p + i) d (mod 2^32) with an odd step d mixed from h,
// one addition per word.  The low 16-bit half of a word feeds node x, the
// high half node x+1.  Every word is uniform when h is (so the rounding stays
// unbiased), and the difference of two words, a multiple of d, is itself
// random.  The draws depend only on (x, y, t, i), so results do not depend
// on how nodes are scheduled, batched or laid out.
__device__ __forceinline__ uint32_t node_seed(int x, int y, long long t) {
    uint32_t h = (uint32_t)x * 0x9E3779B1u;
    h ^= (uint32_t)y * 0x85EBCA77u + 0x632BE5ABu;
    h ^= (uint32_t)t * 0xC2B2AE3Du ^ (uint32_t)((unsigned long long)t >> 32) * 0x27D4EB2Fu;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}
__device__ __forceinline__ uint32_t pair_step(uint32_t h) {
    return ((h ^ (h >> 15)) * 0x2C1B3C6Du) | 1u;
}

// 16-byte vector of V stored elements.
template <int S> struct Vec {
    using ST = Storage<S>;
    union { uint4 raw; typename ST::T e[ST::V]; };
};

template <int S>
__device__ __forceinline__ Vec<S> ld_vec(const typename Storage<S>::T *p) {
    Vec<S> v;
    v.raw = *reinterpret_cast<const uint4 *>(p);
    return v;
}
template <int S>
__device__ __forceinline__ Vec<S> ld_vec_nc(const typename Storage<S>::T *p) {
    Vec<S> v;
    v.raw = __ldg(reinterpret_cast<const uint4 *>(p));
    return v;
}
template <int S>
__device__ __forceinline__ void st_vec(typename Storage<S>::T *p, const Vec<S> &v) {
    *reinterpret_cast<uint4 *>(p) = v.raw;
}

// ---------------------------------------------------------------------------
// Per-lattice constants of the collision (computed in FP64 on the host).
// ---------------------------------------------------------------------------
template <typename C> struct CollConst {
    C rho0;          // reference density of the shift
    // Rest factors and weights by symmetry: index [c != 0] for the 1-D
    // factors, [dcls(i)] (rest, axis, diagonal) for the per-direction values.
    C psi0[2];       // 1-D rest factors: guided Psi_0(0) = 1 - theta, Psi_+-(0) = theta/2;
                     // poly2 W_0 = 1 - theta0, W_+- = theta0 / 2; rounded to C ...
    C psi0_lo[2];    // ... plus the rounding remainder (hi + lo exact to ~2^-48)
    C w[3];          // W_i = Psi_a(0) Psi_b(0) rounded to C ...
    C w_lo[3];       // ... plus the rounding remainder
    C shift[3];      // storage shift s_i (rest equilibrium rounded to C)
    C corr[3];       // W_i rho0 - s_i (exact difference, rounded to C)
    C sum_corr;      // sum_i corr_i
    C sigma;         // 1.5 * 2^e with 2^e >= 32 rho0: split constant of the exact
                     // conserved sums (FP32 storage; see conserved)
    C lam;           // 1 - 1/tau
    C inv_2th2;      // 1 / (2 theta^2), theta = lattice theta (guided) or theta0 (poly2)
    C theta;         // lattice theta (guided) or theta0 (poly2)
};

// ---------------------------------------------------------------------------
// Two FP32 lanes in one 64-bit register pair, computed with the packed
// add/sub/mul/fma.rn.f32x2 instructions of sm_100-class GPUs: each lane is
// rounded exactly as the scalar FP32 operation would round it.  The half
// storage formats collide two nodes per instruction this way.
// ---------------------------------------------------------------------------
struct F2 {
    unsigned long long v;
    __device__ __forceinline__ F2() : v(0ull) {}
    __device__ __forceinline__ explicit F2(unsigned long long r) : v(r) {}
    __device__ __forceinline__ F2(float a, float b) {
        asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(a), "f"(b));
    }
    __device__ __forceinline__ explicit F2(float a) {  // broadcast
        asm("mov.b64 %0, {%1, %1};" : "=l"(v) : "f"(a));
    }
    __device__ __forceinline__ explicit F2(int a) : F2((float)a) {}
    __device__ __forceinline__ explicit F2(double a) : F2((float)a) {}
    __device__ __forceinline__ float lo() const {
        float a;
        asm("mov.b64 {%0, _}, %1;" : "=f"(a) : "l"(v));
        return a;
    }
    __device__ __forceinline__ float hi() const {
        float b;
        asm("mov.b64 {_, %0}, %1;" : "=f"(b) : "l"(v));
        return b;
    }
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    F2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2(0.0f) - a; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) {
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
using ::fma;  // keep the scalar overloads visible next to the packed one

// Per-lane IEEE division (the packed reciprocal estimate plus a Newton step
// measured 15% slower in the half-format kernels).
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.lo() / b.lo(), a.hi() / b.hi()); }

// Error-free sum: a + b = s + e exactly (Knuth TwoSum).
template <typename C>
__device__ __forceinline__ void two_sum(C a, C b, C &s, C &e) {
    s = a + b;
    C bp = s - a;
    C ap = s - bp;
    e = (a - ap) + (b - bp);
}

// Rounded addition and subtraction that the compiler may neither contract nor
// reassociate (the split below relies on every intermediate rounding).
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
// packed pairs: each lane rounds as the scalar FP32 operation (inline PTX,
// which the compiler does not reassociate)
__device__ __forceinline__ F2 add_rn(F2 a, F2 b) { return a + b; }
__device__ __forceinline__ F2 sub_rn(F2 a, F2 b) { return a - b; }

// Conserved moments of one node from its shifted populations g.
//   drho = rho - rho0 = sum g_i - sum corr_i,  j = sum c_i g_i
// (the shifts cancel in j because opposite directions share one shift).
//
// The constant sum_corr (the shifts' rounding remainders, ~1e-8) enters the
// sum first: subtracted last, it falls below half a unit of drho wherever
// |rho - rho0| is large and is rounded away identically at every node and
// step, a steady mass loss that dominates the drift of long FP32 runs.
//
// EXACT (FP32 storage) makes the sums exact, rounded once.  Each g_i splits
// error-free into q_i = (g_i + sigma) - sigma, g_i rounded to the grid
// ulp(sigma) = 2^(e-23), and r_i = g_i - q_i, |r_i| <= ulp(sigma) / 2.  While
// |g_i| < 2^(e-1) (sigma = 1.5 * 2^e) the q_i and every partial sum of up to
// nine of them (below 2^(e+1)) lie on the grid, so the q sums carry no
// rounding; the r sums round at ~2^-24 of their size, ~2^(e-45).  drho and j
// are then the exact sums up to one final rounding.  With 2^e >= 32 rho0 the
// sums are exact for |g_i| < 7 rho0; beyond that they degrade to ordinary
// rounded sums.  On the 2048 x 4 shock tube (tau = 0.51, 2000 steps) the
// plain FP32 sums end 3e-5 from the FP64 scheme, these 1e-6..5e-6.
template <typename C, bool EXACT>
__device__ __forceinline__ void conserved(const C g[9], const CollConst<C> &k, C &drho,
                                          C &jx, C &jy) {
    if constexpr (!EXACT) {
        drho = (((g[0] - k.sum_corr) + (g[1] + g[2])) + ((g[3] + g[4]) + (g[5] + g[6]))) +
               (g[7] + g[8]);
        jx = ((g[1] - g[3]) + (g[5] - g[6])) + (g[8] - g[7]);
        jy = ((g[2] - g[4]) + (g[5] + g[6])) - (g[7] + g[8]);
    } else {
        // accumulated direction by direction, so that only the six partial
        // sums stay live
        C q, r, qd, rd, qx, rx, qy, ry;
        auto split = [&](C gi) {
            q = sub_rn(add_rn(gi, k.sigma), k.sigma);
            r = sub_rn(gi, q);
        };
        split(g[0]); qd = q; rd = r - k.sum_corr;
        split(g[1]); qd = qd + q; rd = rd + r; qx = q; rx = r;
        split(g[2]); qd = qd + q; rd = rd + r; qy = q; ry = r;
        split(g[3]); qd = qd + q; rd = rd + r; qx = qx - q; rx = rx - r;
        split(g[4]); qd = qd + q; rd = rd + r; qy = qy - q; ry = ry - r;
        split(g[5]); qd = qd + q; rd = rd + r; qx = qx + q; rx = rx + r; qy = qy + q; ry = ry + r;
        split(g[6]); qd = qd + q; rd = rd + r; qx = qx - q; rx = rx - r; qy = qy + q; ry = ry + r;
        split(g[7]); qd = qd + q; rd = rd + r; qx = qx - q; rx = rx - r; qy = qy - q; ry = ry - r;
        split(g[8]); qd = qd + q; rd = rd + r; qx = qx + q; rx = rx + r; qy = qy - q; ry = ry - r;
        drho = qd + rd;
        jx = qx + rx;
        jy = qy + ry;
    }
}

// One node's collision in shifted variables: g (pre-collision, f - s) in,
// post (post-collision, f - s) out.
//
// Moments: rho = rho0 + drho, u = j / rho; the trace-free non-equilibrium
// stress of Eq. 6's inner sum, S_ab = sum_k (c_ka c_kb - c_k^2 delta_ab / 2)
// f^neq_k, equals Pi - Pi^eq with Pi^eq = rho theta delta + rho u u for both
// equilibria, so S_xx = ((Pi_xx - Pi_yy) - rho (u_x^2 - u_y^2)) / 2 and
// S_xy = Pi_xy - rho u_x u_y (the shifts cancel in Pi_xx - Pi_yy and Pi_xy).
// Equilibrium deviation geq_i = f^eq_i - s_i:
//   guided (Eq. 11, f^eq = rho Psi_a(u_x) Psi_b(u_y)):
//     geq = drho W + rho (dPsi_a Psi_b + Psi_a(0) dPsi_b) + corr, with
//     dPsi_0 = -u^2, dPsi_+- = (+-u + u^2)/2;
//   poly2 (Eq. 15): geq = W (drho + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u^2)) + corr.
// OReg (Eqs. 6, 7): f^OReg_i = f^eq_i / (2 rho theta^2)
//   [(C_x^2 - C_y^2) S_xx + 2 C_x C_y S_xy], C = c - u (the delta terms of
// Eq. 6 vanish because S is trace-free), post = geq + (1 - 1/tau) f^OReg.
// BGK (Eq. 1): post = geq + (1 - 1/tau) (g - geq).
//
// HAVE_MOM: drho, jx, jy come in as mom[0..2] (the FP32 kernels form the exact
// sums of two nodes at once with packed arithmetic; see collide_vec).
template <int EQ, int COLL, typename C, bool EXACT, bool HAVE_MOM = false>
__device__ __forceinline__ void collide(const C g[9], C post[9], const CollConst<C> &k,
                                        const C *mom = nullptr) {
    // Packed pairs (issue-bound half formats) share the opposite-direction
    // sums between the conserved moments and the stress and fold the OReg
    // prefactor into the stress; float and double keep the plain order.
    constexpr bool PACKED = std::is_same<C, F2>::value;
    constexpr bool LOCAL = EQ == EQ_GUIDED_LOCAL;
    C drho, jx, jy, dxy, pxy, tg = C(0);
    if constexpr (HAVE_MOM) {
        drho = mom[0];
        jx = mom[1];
        jy = mom[2];
        dxy = (g[1] + g[3]) - (g[2] + g[4]);
        pxy = (g[5] + g[7]) - (g[6] + g[8]);
        if constexpr (LOCAL) tg = ((g[1] + g[3]) + (g[2] + g[4])) + C(2) * ((g[5] + g[7]) + (g[6] + g[8]));
    } else if constexpr (PACKED && !EXACT) {
        const C s13 = g[1] + g[3], s24 = g[2] + g[4], s57 = g[5] + g[7], s68 = g[6] + g[8];
        const C d13 = g[1] - g[3], d24 = g[2] - g[4], d57 = g[5] - g[7], d68 = g[6] - g[8];
        drho = (((g[0] - k.sum_corr) + s13) + (s24 + s57)) + s68;
        jx = (d13 + d57) - d68;
        jy = (d24 + d57) + d68;
        dxy = s13 - s24;
        pxy = s57 - s68;
        if constexpr (LOCAL) tg = (s13 + s24) + C(2) * (s57 + s68);
    } else {
        conserved<C, EXACT>(g, k, drho, jx, jy);
        dxy = (g[1] + g[3]) - (g[2] + g[4]);
        pxy = (g[5] + g[7]) - (g[6] + g[8]);
        if constexpr (LOCAL) tg = ((g[1] + g[3]) + (g[2] + g[4])) + C(2) * ((g[5] + g[7]) + (g[6] + g[8]));
    }
    // Scalar FP32 (UNBIASED): no rounding that repeats identically at every
    // node may enter the update.  rho = rho0 + drho rounds to the same float
    // wherever rho is near rho0, and so does 1/rho: products with the rounded
    // rho or 1/rho carry a relative error of up to 2^-24 that is the same
    // everywhere, a per-step bias of ~1e-8 that a slowly decaying shear wave
    // (decay ~1e-5 per step) turns into a decay-rate error of 1e-4..4e-4.  So
    // rho enters products as rho0 x + drho x, and 1/rho carries the residual
    // of its rounding against rho0 + drho.
    constexpr bool UNBIASED = std::is_same<C, float>::value;
    const C rho = k.rho0 + drho;
    const C inv_rho = C(1) / rho;
    C inv_lo = C(0);
    if constexpr (UNBIASED)
        inv_lo = fma(-drho, inv_rho, fma(-k.rho0, inv_rho, C(1))) * inv_rho;
    auto rho_times = [&](C x) { return UNBIASED ? fma(drho, x, k.rho0 * x) : rho * x; };
    const C ux = UNBIASED ? fma(jx, inv_rho, jx * inv_lo) : jx * inv_rho;
    const C uy = UNBIASED ? fma(jy, inv_rho, jy * inv_lo) : jy * inv_rho;
    const C ux2 = ux * ux, uy2 = uy * uy;
    // Local temperature (EQ_GUIDED_LOCAL): 2 rho theta = <f,c^2> - rho u^2
    // (Eq. 2a energy), written as theta = theta_ref + dth with
    // 2 rho dth = sum c^2 g - sum c^2 corr - 2 theta_ref drho - rho u^2, all
    // small deviations (the shifts' own sum c^2 s = 2 theta_ref rho0 - sum
    // c^2 corr cancels exactly).  Psi_0 = 1 - theta - u^2 and
    // Psi_+- = (theta +- u + u^2)/2 then deviate from their rest values at
    // theta_ref by dth as well as by u.
    C dth = C(0);
    if constexpr (LOCAL) {
        const C c2corr = C(4) * k.corr[1] + C(8) * k.corr[2];
        dth = C(0.5) * inv_rho *
              (((tg - c2corr) - C(2) * k.theta * drho) - rho * (ux2 + uy2));
    }

    // The equilibrium constants enter in hi + lo form.  Rounded to C alone
    // they would break sum_b Psi_b(0) = 1 and sum_i W_i c_i c_i = theta by a
    // unit roundoff, which acts as a small mass and momentum source on every
    // node at every step; in FP32 that bias, not random rounding, dominates
    // the drift from the FP64 result over thousands of steps.
    C geq[9];
    if constexpr (EQ == EQ_GUIDED || LOCAL) {
        // dPsi_+- = u^2/2 +- u/2, dPsi_0 = -u^2 (u/2 and u^2/2 are exact halvings);
        // with the local temperature u^2 -> u^2 + dth
        const C ex2 = LOCAL ? ux2 + dth : ux2, ey2 = LOCAL ? uy2 + dth : uy2;
        const C qx = C(0.5) * ux, hx = C(0.5) * ex2, qy = C(0.5) * uy, hy = C(0.5) * ey2;
        const C dpx[3] = {-ex2, hx + qx, hx - qx};
        const C dpy[3] = {-ey2, hy + qy, hy - qy};
        // packed (issue-bound) path: drho W_lo + corr once per symmetry class;
        // the scalar path keeps it per direction (fewer live registers, which
        // the HBM-bound FP32 in-place kernels need for occupancy)
        C c3[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) c3[c] = PACKED ? fma(drho, k.w_lo[c], k.corr[c]) : k.corr[c];
        // UNBIASED: the shift correction corr (below half a unit of geq) is
        // added inside the sum that forms t, as corr / rho, so that it is
        // rounded together with the exact value; added to the already
        // rounded rho t it would be rounded away alike at every node.
        C cr[3] = {C(0), C(0), C(0)};
        if constexpr (UNBIASED) {
#pragma unroll
            for (int c = 0; c < 3; ++c) cr[c] = k.corr[c] * (inv_rho + inv_lo);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int a = kidx(cx_of(i)), b = kidx(cy_of(i));
            const int pa = cx_of(i) != 0, pb = cy_of(i) != 0, ci = dcls(i);
            // dPsi_a Psi_b + Psi_a(0) dPsi_b with Psi(0) = hi + lo
            const C psib = k.psi0[pb] + dpy[b];
            const C t = fma(dpx[a], psib,
                            fma(dpx[a], k.psi0_lo[pb],
                                fma(k.psi0[pa], dpy[b],
                                    UNBIASED ? fma(k.psi0_lo[pa], dpy[b], cr[ci])
                                             : k.psi0_lo[pa] * dpy[b])));
            if constexpr (PACKED) {
                geq[i] = fma(drho, k.w[ci], fma(rho, t, c3[ci]));
            } else {
                const C vel = UNBIASED ? rho_times(t) : fma(rho, t, k.corr[ci]);
                geq[i] = fma(drho, k.w[ci], fma(drho, k.w_lo[ci], vel));
            }
        }
    } else {
        const C u2 = ux2 + uy2;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const C cu = C(cx_of(i)) * ux + C(cy_of(i)) * uy;
            const C poly = fma(C(3), cu, fma(C(4.5) * cu, cu, C(-1.5) * u2));
            const C rp = rho_times(poly);
            const int ci = dcls(i);
            const C vel = fma(rp, k.w[ci], fma(rp, k.w_lo[ci], k.corr[ci]));
            geq[i] = fma(drho, k.w[ci], fma(drho, k.w_lo[ci], vel));
        }
    }

    if constexpr (COLL == COLL_BGK) {
#pragma unroll
        for (int i = 0; i < 9; ++i) post[i] = fma(k.lam, g[i] - geq[i], geq[i]);
    } else {
        const C sxx = C(0.5) * (dxy - rho_times(ux2 - uy2));
        const C sxy = pxy - rho_times(ux * uy);
        C a;
        if constexpr (LOCAL) {
            const C th = k.theta + dth;
            a = k.lam / (C(2) * th * th * rho);
        } else {
            a = k.lam * k.inv_2th2 * (UNBIASED ? inv_rho + inv_lo : inv_rho);
        }
        const C X[3] = {-ux, C(1) - ux, C(-1) - ux};
        const C Y[3] = {-uy, C(1) - uy, C(-1) - uy};
        if constexpr (PACKED) {
            // a d_i expanded in c_i (an identity of the contraction below):
            //   a d_i = A + Sxx (cx^2 - cy^2) + 2 Sxy cx cy - cx P + cy Q, with
            //   Sxx = a sxx, Sxy = a sxy, A = Sxx (ux^2 - uy^2) + 2 Sxy ux uy,
            //   P = 2 (Sxx ux + Sxy uy), Q = 2 (Sxx uy - Sxy ux),
            // so each direction costs one or two additions.
            const C Sxx = a * sxx, Sxy = a * sxy, Sxy2 = C(2) * Sxy;
            const C A = fma(Sxx, ux2 - uy2, Sxy2 * (ux * uy));
            const C P = C(2) * fma(Sxx, ux, Sxy * uy), Q = C(2) * fma(Sxx, uy, -(Sxy * ux));
            const C Ap = A + Sxx, Am = A - Sxx, Dp = A + Sxy2, Dm = A - Sxy2;
            C ad[9];
            ad[0] = A;
            ad[1] = Ap - P;            // (+1, 0)
            ad[3] = Ap + P;            // (-1, 0)
            ad[2] = Am + Q;            // (0, +1)
            ad[4] = Am - Q;            // (0, -1)
            ad[5] = (Dp - P) + Q;      // (+1, +1)
            ad[7] = (Dp + P) - Q;      // (-1, -1)
            ad[6] = (Dm + P) + Q;      // (-1, +1)
            ad[8] = (Dm - P) - Q;      // (+1, -1)
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const C feq = k.shift[dcls(i)] + geq[i];
                post[i] = fma(feq, ad[i], geq[i]);
            }
        } else {
            const C two_sxy = C(2) * sxy;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int ia = kidx(cx_of(i)), ib = kidx(cy_of(i));
                const C d = fma(X[ia] * X[ia] - Y[ib] * Y[ib], sxx, X[ia] * Y[ib] * two_sxy);
                const C feq = k.shift[dcls(i)] + geq[i];
                post[i] = fma(feq, a * d, geq[i]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Warp-level shifted row access.
//
// Each lane owns V consecutive nodes x = xb .. xb+V-1 of one row.  Row
// storage has a pitch that is a multiple of V, so a lane's V elements are one
// aligned 16-byte vector.  Shuffles run within groups of W lanes (sub = the
// lane's index in its group) whose vectors are consecutive within a row, except
// where a row begins (xb = 0) or ends (xb + V >= nx): there the neighbour
// comes from memory (halo and wrap elements).  The stream-collide kernels use
// one group of 32 lanes holding 32 consecutive vectors of a plane in
// row-major order, which may span rows.  Lanes with xb >= nx are idle but
// still take part in the shuffles.
// ---------------------------------------------------------------------------

// Pull, in two phases so that a warp has all nine row fetches in flight
// before it uses any of them:
//   fetch_row: the lane's 16-byte vector at xb plus the one halo element the
//              shift needs from outside the warp (or across the periodic wrap);
//   shift_row: decode and move each value one node along x with shuffles, so
//              that out[j] = value at x - CX (periodic) of node x = xb + j.
// NC selects the read-only data path (A-B layout).
template <int S> struct RawRow {
    Vec<S> v;
    typename Storage<S>::T halo;  // left (CX = +1) or right (CX = -1) neighbour
    typename Storage<S>::T wrap;  // CX = -1: value at x = 0 for node nx - 1
};

template <int S, int CX, bool NC>
__device__ __forceinline__ RawRow<S> fetch_row(const typename Storage<S>::T *rowp, int xb, int nx,
                                               int sub, int W) {
    using ST = Storage<S>;
    constexpr int V = ST::V;
    RawRow<S> r;
    r.v.raw = make_uint4(0, 0, 0, 0);
    r.halo = typename ST::T(0.0f);
    r.wrap = typename ST::T(0.0f);
    if (xb < nx) {
        r.v = NC ? ld_vec_nc<S>(rowp + xb) : ld_vec<S>(rowp + xb);
        if constexpr (CX == 1) {
            if (sub == 0 || xb == 0) r.halo = rowp[xb == 0 ? nx - 1 : xb - 1];
        } else if constexpr (CX == -1) {
            if (sub == W - 1 && xb + V < nx) r.halo = rowp[xb + V];
            if (xb + V >= nx) r.wrap = rowp[0];
        }
    }
    return r;
}

template <int S, int CX>
__device__ __forceinline__ void shift_row(const RawRow<S> &r, int xb, int nx, int sub, int W,
                                          typename Storage<S>::C out[Storage<S>::V]) {
    using ST = Storage<S>;
    using C = typename ST::C;
    constexpr int V = ST::V;
    C a[V];
#pragma unroll
    for (int j = 0; j < V; ++j) a[j] = ST::dec_step(r.v.e[j]);
    if constexpr (CX == 0) {
#pragma unroll
        for (int j = 0; j < V; ++j) out[j] = a[j];
    } else if constexpr (CX == 1) {
        // left neighbour of the lane's first node
        C left = __shfl_up_sync(0xffffffffu, a[V - 1], 1, W);
        if (xb < nx && (sub == 0 || xb == 0)) left = ST::dec_step(r.halo);
        out[0] = left;
#pragma unroll
        for (int j = 1; j < V; ++j) out[j] = a[j - 1];
    } else {
        // right neighbour of the lane's last node; node nx-1 wraps to x = 0
        C right = __shfl_down_sync(0xffffffffu, a[0], 1, W);
        if (xb < nx && sub == W - 1 && xb + V < nx) right = ST::dec_step(r.halo);
        const C wrapv = ST::dec_step(r.wrap);
#pragma unroll
        for (int j = 0; j < V - 1; ++j) out[j] = a[j + 1];
        out[V - 1] = right;
#pragma unroll
        for (int j = 0; j < V; ++j)
            if (xb + j == nx - 1) out[j] = wrapv;
    }
}

// Shuffles of raw stored elements (2, 4 or 8 bytes).
template <typename T>
__device__ __forceinline__ T shfl_up_raw(T v, int d, int w) {
    if constexpr (sizeof(T) == 2) {
        unsigned short b;
        memcpy(&b, &v, 2);
        b = (unsigned short)__shfl_up_sync(0xffffffffu, (unsigned)b, d, w);
        memcpy(&v, &b, 2);
        return v;
    } else {
        return __shfl_up_sync(0xffffffffu, v, d, w);
    }
}
template <typename T>
__device__ __forceinline__ T shfl_down_raw(T v, int d, int w) {
    if constexpr (sizeof(T) == 2) {
        unsigned short b;
        memcpy(&b, &v, 2);
        b = (unsigned short)__shfl_down_sync(0xffffffffu, (unsigned)b, d, w);
        memcpy(&v, &b, 2);
        return v;
    } else {
        return __shfl_down_sync(0xffffffffu, v, d, w);
    }
}

// Stores of part of a lane's 16-byte vector at p (16-byte aligned), in pieces
// aligned to their size: the elements 1 .. V-1, or the first L (0 <= L < V).
template <int S>
__device__ __forceinline__ void st_tail1(typename Storage<S>::T *p, const Vec<S> &v) {
    constexpr int V = Storage<S>::V;
    char *b = reinterpret_cast<char *>(p);
    if constexpr (V == 2) {
        *reinterpret_cast<uint2 *>(b + 8) = make_uint2(v.raw.z, v.raw.w);
    } else if constexpr (V == 4) {
        *reinterpret_cast<unsigned *>(b + 4) = v.raw.y;
        *reinterpret_cast<uint2 *>(b + 8) = make_uint2(v.raw.z, v.raw.w);
    } else {
        *reinterpret_cast<unsigned short *>(b + 2) = (unsigned short)(v.raw.x >> 16);
        *reinterpret_cast<unsigned *>(b + 4) = v.raw.y;
        *reinterpret_cast<uint2 *>(b + 8) = make_uint2(v.raw.z, v.raw.w);
    }
}
template <int S>
__device__ __forceinline__ void st_head(typename Storage<S>::T *p, const Vec<S> &v, int L) {
    constexpr int V = Storage<S>::V;
    char *b = reinterpret_cast<char *>(p);
    if constexpr (V == 2) {
        if (L & 1) *reinterpret_cast<uint2 *>(b) = make_uint2(v.raw.x, v.raw.y);
    } else if constexpr (V == 4) {
        if (L & 2) *reinterpret_cast<uint2 *>(b) = make_uint2(v.raw.x, v.raw.y);
        if (L & 1) *reinterpret_cast<unsigned *>(b + 4 * (L & 2)) = (L & 2) ? v.raw.z : v.raw.x;
    } else {
        if (L & 4) *reinterpret_cast<uint2 *>(b) = make_uint2(v.raw.x, v.raw.y);
        if (L & 2) *reinterpret_cast<unsigned *>(b + 2 * (L & 4)) = (L & 4) ? v.raw.z : v.raw.x;
        if (L & 1) {
            const int k = L & 6;
            const unsigned w = (k & 4) ? ((k & 2) ? v.raw.w : v.raw.z) : ((k & 2) ? v.raw.y : v.raw.x);
            *reinterpret_cast<unsigned short *>(b + 2 * k) = (unsigned short)(w & 0xFFFFu);
        }
    }
}
// Element j (0 <= j < V) of a lane's vector, as raw bits of the element size.
template <int S>
__device__ __forceinline__ typename Storage<S>::T vec_elem(const Vec<S> &v, int j) {
    constexpr int V = Storage<S>::V;
    using T = typename Storage<S>::T;
    T out;
    if constexpr (V == 2) {
        const uint2 w = (j & 1) ? make_uint2(v.raw.z, v.raw.w) : make_uint2(v.raw.x, v.raw.y);
        memcpy(&out, &w, 8);
    } else if constexpr (V == 4) {
        const unsigned w = (j & 2) ? ((j & 1) ? v.raw.w : v.raw.z) : ((j & 1) ? v.raw.y : v.raw.x);
        memcpy(&out, &w, 4);
    } else {
        const unsigned w = (j & 4) ? ((j & 2) ? v.raw.w : v.raw.z) : ((j & 2) ? v.raw.y : v.raw.x);
        const unsigned short h = (unsigned short)((j & 1) ? (w >> 16) : (w & 0xFFFFu));
        memcpy(&out, &h, 2);
    }
    return out;
}

// Push of already encoded elements: e[j] of node x = xb + j goes to position
// x + CX (periodic) of the row at rowp.  Each position is written exactly
// once, by the lane that owns the node the value comes from; positions past
// nx (row padding) may receive any of the lane's values.
template <int S, int CX>
__device__ __forceinline__ void store_row_shifted_raw(typename Storage<S>::T *rowp, int xb, int nx,
                                                      int sub, int W,
                                                      const typename Storage<S>::T e[Storage<S>::V]) {
    using T = typename Storage<S>::T;
    constexpr int V = Storage<S>::V;
    const bool active = xb < nx;
    if constexpr (CX == 0) {
        if (active) {
            Vec<S> v;
#pragma unroll
            for (int j = 0; j < V; ++j) v.e[j] = e[j];
            st_vec<S>(rowp + xb, v);
        }
    } else if constexpr (CX == 1) {
        const T from_left = shfl_up_raw(e[V - 1], 1, W);
        if (active) {
            Vec<S> v;
            v.e[0] = from_left;
#pragma unroll
            for (int j = 1; j < V; ++j) v.e[j] = e[j - 1];
            // element 0 of a lane that starts the warp or the row comes from
            // another lane's push (the warp's neighbour, or the row's end)
            if (!(sub == 0 || xb == 0)) st_vec<S>(rowp + xb, v);
            else st_tail1<S>(rowp + xb, v);
            // node nx - 1 wraps to x = 0: it is element nx - 1 - xb of v shifted by one
            if (xb + V > nx - 1) {
                Vec<S> o;
#pragma unroll
                for (int j = 0; j < V; ++j) o.e[j] = e[j];
                rowp[0] = vec_elem<S>(o, nx - 1 - xb);
            }
            if (sub == W - 1 && xb + V < nx) rowp[xb + V] = e[V - 1];
        }
    } else {
        const T from_right = shfl_down_raw(e[0], 1, W);
        if (active) {
            Vec<S> v;
#pragma unroll
            for (int j = 0; j < V - 1; ++j) v.e[j] = e[j + 1];
            v.e[V - 1] = from_right;
            // a lane holding the row's end writes x = xb .. nx - 2 (x = nx - 1
            // gets node 0's value); the warp's last lane leaves its last
            // element to the next warp's first lane
            const bool has_row_end = xb + V > nx - 1;
            const bool last_foreign = (sub == W - 1) && (xb + V < nx);
            if (!has_row_end && !last_foreign) st_vec<S>(rowp + xb, v);
            else st_head<S>(rowp + xb, v, has_row_end ? nx - 1 - xb : V - 1);
            if (xb == 0) rowp[nx - 1] = e[0];
            else if (sub == 0) rowp[xb - 1] = e[0];
        }
    }
}

__device__ __forceinline__ int wrap_row(int y, int ny) {
    return y < 0 ? y + ny : (y >= ny ? y - ny : y);
}

}  // namespace oreg
