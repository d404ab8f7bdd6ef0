// Host-side construction of the collision constants (CollConst) of a lattice
// from its olb_params, shared by every unit that needs a lattice's shifts:
// the lattice objects (oreg_api.cu) and the no-allocation reduction
// (oreg_noalloc.cu).
#pragma once

#include <cmath>

#include "oreg.h"
#include "oreg_device.cuh"

namespace oreg {

// hi + lo split of a double into the compute type C: hi = (C)v and lo the
// remainder, so that hi + lo represents v to ~2^-48 in FP32.
template <typename C>
inline void split(double v, C &hi, C &lo) {
    hi = (C)v;
    lo = (C)(v - (double)hi);
}

// Constants of the collision for the compute type C.  The storage shift s_i
// is the rest equilibrium w_i rho0 rounded to C and corr_i the exact
// remainder w_i rho0 - s_i; the rest factors and weights are kept as hi + lo
// pairs (see collide()).
template <typename C>
inline CollConst<C> make_const(const olb_params *p) {
    CollConst<C> k;
    const double th = p->eq == OLB_EQ_GUIDED ? p->theta : 1.0 / 3.0;
    const double psi0[2] = {1.0 - th, 0.5 * th};
    for (int a = 0; a < 2; ++a) split<C>(psi0[a], k.psi0[a], k.psi0_lo[a]);
    // classes: rest (psi0 psi0), axis (psi0 psi+-), diagonal (psi+- psi+-)
    const double w[3] = {psi0[0] * psi0[0], psi0[0] * psi0[1], psi0[1] * psi0[1]};
    const int count[3] = {1, 4, 4};
    double corr_sum = 0.0;
    for (int c = 0; c < 3; ++c) {
        split<C>(w[c], k.w[c], k.w_lo[c]);
        const C s = (C)(w[c] * p->rho0);
        const double corr = w[c] * p->rho0 - (double)s;
        k.shift[c] = s;
        k.corr[c] = (C)corr;
        corr_sum += count[c] * corr;
    }
    k.sum_corr = (C)corr_sum;
    k.rho0 = (C)p->rho0;
    // split constant of the exact conserved sums: 1.5 * 2^e, 2^e >= 32 rho0
    k.sigma = (C)(1.5 * std::exp2(std::ceil(std::log2(32.0 * p->rho0))));
    k.lam = (C)(1.0 - 1.0 / p->tau);
    k.inv_2th2 = (C)(1.0 / (2.0 * th * th));
    k.theta = (C)th;
    return k;
}

// FP32 constants of the stream-collide kernels, in the storage format's step
// units (populations, rho0, shifts and corrections times STEP_SCALE, a power
// of two; see Storage in oreg_device.cuh).
inline CollConst<float> make_step_const_f32(const olb_params *p) {
    olb_params q = *p;
    if (p->storage == OLB_F16_SHIFTED) q.rho0 *= Storage<ST_F16>::STEP_SCALE;
    return make_const<float>(&q);
}

// FP64 constants (initialisation and readback) whose shift is exactly the
// stored format's shift.
inline CollConst<double> make_const_f64_for(const olb_params *p) {
    CollConst<double> kd = make_const<double>(p);
    if (p->storage != OLB_F64) {
        const CollConst<float> kf = make_const<float>(p);
        const int count[3] = {1, 4, 4};
        double corr_sum = 0.0;
        for (int c = 0; c < 3; ++c) {
            kd.shift[c] = (double)kf.shift[c];
            kd.corr[c] = kd.w[c] * p->rho0 - kd.shift[c];
            corr_sum += count[c] * kd.corr[c];
        }
        kd.sum_corr = corr_sum;
    }
    return kd;
}

}  // namespace oreg
