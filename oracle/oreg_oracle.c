/*
 * Plain FP64 CPU oracle for the Onsager-Regularized (OReg) lattice Boltzmann
 * update on D2Q9 (Jonnalagadda et al., arXiv 2501.16000).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal statement of the
 * scheme that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Every routine follows one passage of the paper, written out as the paper
 * states it (no algebraic shortcuts), in double precision, compiled without
 * floating-point contraction:
 *
 *   ora_feq            Eq. 11 (guided equilibrium, as printed) and Eq. 15
 *                      (second-order polynomial equilibrium; the printed form
 *                      lacks the -u^2/(2 theta0) term, which is restored so
 *                      that Eq. 2a holds).
 *   ora_foreg          Eq. 6 (local OReg populations), with both alpha,beta
 *                      double sums and both delta terms kept.
 *   ora_collide_node   Eq. 7 (OReg update) or Eq. 1 (lattice BGK).
 *   ora_stream         left-hand side of Eqs. 1 and 7: the post-collision
 *                      population i at x lands at x + c_i (periodic).
 *   ora_step           one full time step = collide at every node, then stream.
 *   ora_bounce_back_node  full-way bounce-back at the wall nodes of the Sec. IV
 *                      shock tube (post_i = f_opp(i)).
 *   ora_first_order    Eq. 5 (first-order populations from a velocity
 *                      gradient), used to start a run without the transient
 *                      of an equilibrium start.
 *
 * Parity status: pinned by the closed forms of Eqs. 2, 12, 13, 16 and 17, by
 * streaming translation, conservation, the viscous shear-wave decay of
 * Eq. 14a and the isothermal Riemann problem (tests/test_oracle_pins.py).
 *
 * State layout: f[(i*ny + y)*nx + x], i = 0..8 in the velocity order below,
 * the canonical pre-collision populations at integer time t.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_Q 9
#define ORA_D 2

/* D2Q9 velocity set c_i in {-1,0,1}^2 (Fig. 1a). */
static const int ORA_C[ORA_Q][ORA_D] = {
    {0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};

typedef struct {
    int32_t nx, ny;
    double tau;
    double theta;     /* lattice temperature used by the guided equilibrium */
    int32_t eq;       /* 0 = guided (Eq. 11), 1 = polynomial (Eq. 15) */
    int32_t coll;     /* 0 = OReg (Eq. 7), 1 = BGK (Eq. 1) */
    int32_t walls;    /* 1: columns x = 0 and x = nx - 1 are full-way
                         bounce-back walls (Sec. IV shock tube); 0: periodic */
    int32_t theta_local; /* guided only.  0: theta is the fixed lattice
                            temperature (isothermal, Sec. II); 1: each node's
                            equilibrium and Eq. 6 use the node's own
                            temperature (<f,c^2> - rho u^2) / (D rho) */
} ora_params;

/* Reference temperature of the polynomial equilibrium (Eq. 15). */
static const double ORA_THETA0 = 1.0 / 3.0;

int ora_q(void) { return ORA_Q; }

void ora_velocities(int32_t *out /* [9][2] */) {
    for (int i = 0; i < ORA_Q; ++i) {
        out[2 * i] = ORA_C[i][0];
        out[2 * i + 1] = ORA_C[i][1];
    }
}

void ora_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int ora_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Temperature entering Eq. 6: the lattice theta for the guided equilibrium,
 * theta0 = 1/3 for the polynomial equilibrium, which is only defined there. */
static double ora_theta_eff(int eq, double theta) {
    return eq == 0 ? theta : ORA_THETA0;
}

/* Eq. 11 written as printed: for each axis alpha,
 *   (1 - 2 c_a^2) / 2^(c_a^2) * [c_a^2 - 1 + c_a u_a + u_a^2 + theta],
 * multiplied over alpha = x, y and by rho.
 * Eq. 15 with weights W = prod_a W_{c_a}, W_0 = 1 - theta0, W_{+-1} = theta0/2:
 *   rho W_i [1 + (c_i.u)/theta0 + (c_i.u)^2/(2 theta0^2) - u.u/(2 theta0)]. */
void ora_feq(int eq, double theta, double rho, double ux, double uy,
             double *feq /* [9] */) {
    const double u[ORA_D] = {ux, uy};
    for (int i = 0; i < ORA_Q; ++i) {
        if (eq == 0) {
            double prod = rho;
            for (int a = 0; a < ORA_D; ++a) {
                const double c = (double)ORA_C[i][a];
                const double c2 = c * c;
                const double factor = (1.0 - 2.0 * c2) / pow(2.0, c2);
                prod *= factor * (c2 - 1.0 + c * u[a] + u[a] * u[a] + theta);
            }
            feq[i] = prod;
        } else {
            const double t0 = ORA_THETA0;
            double W = 1.0;
            for (int a = 0; a < ORA_D; ++a)
                W *= (ORA_C[i][a] == 0) ? (1.0 - t0) : (t0 / 2.0);
            double cu = 0.0, uu = 0.0;
            for (int a = 0; a < ORA_D; ++a) {
                cu += (double)ORA_C[i][a] * u[a];
                uu += u[a] * u[a];
            }
            feq[i] = rho * W *
                     (1.0 + cu / t0 + (cu * cu) / (2.0 * t0 * t0) - uu / (2.0 * t0));
        }
    }
}

/* Density and velocity of one node: rho = <f,1>, rho u = <f,c> (Eq. 2a). */
void ora_node_moments(const double *f, double *rho, double *ux, double *uy) {
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < ORA_Q; ++i) {
        r += f[i];
        jx += (double)ORA_C[i][0] * f[i];
        jy += (double)ORA_C[i][1] * f[i];
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
}

/* Eq. 6: f_i^OReg = f_i^eq / (2 rho theta^2)
 *                   * sum_{a,b} (C_ia C_ib - C_i^2 delta_ab / D)
 *                               * sum_k (c_ka c_kb - c_k^2 delta_ab / D) f_k^neq,
 * with C_i = c_i - u, f^neq = f - f^eq (the predictor of Sec. II) and D = 2.
 * The inner sum over k does not depend on i; it is formed once per node. */
void ora_foreg(const double *f, const double *feq, double rho, double ux, double uy,
               double theta_eff, double *foreg /* [9] */) {
    const double u[ORA_D] = {ux, uy};
    double fneq[ORA_Q];
    for (int k = 0; k < ORA_Q; ++k) fneq[k] = f[k] - feq[k];

    double S[ORA_D][ORA_D];
    for (int a = 0; a < ORA_D; ++a) {
        for (int b = 0; b < ORA_D; ++b) {
            double s = 0.0;
            for (int k = 0; k < ORA_Q; ++k) {
                const double ca = (double)ORA_C[k][a], cb = (double)ORA_C[k][b];
                const double ck2 = (double)(ORA_C[k][0] * ORA_C[k][0] + ORA_C[k][1] * ORA_C[k][1]);
                const double delta = (a == b) ? 1.0 : 0.0;
                s += (ca * cb - ck2 * delta / (double)ORA_D) * fneq[k];
            }
            S[a][b] = s;
        }
    }

    for (int i = 0; i < ORA_Q; ++i) {
        double C[ORA_D];
        for (int a = 0; a < ORA_D; ++a) C[a] = (double)ORA_C[i][a] - u[a];
        const double C2 = C[0] * C[0] + C[1] * C[1];
        double contraction = 0.0;
        for (int a = 0; a < ORA_D; ++a) {
            for (int b = 0; b < ORA_D; ++b) {
                const double delta = (a == b) ? 1.0 : 0.0;
                contraction += (C[a] * C[b] - C2 * delta / (double)ORA_D) * S[a][b];
            }
        }
        foreg[i] = feq[i] / (2.0 * rho * theta_eff * theta_eff) * contraction;
    }
}

/* Temperature of one node's populations: E = <f, c^2/2> = (D p + rho u^2)/2
 * with p = rho theta (Eq. 2a and the definitions after Eq. 2), solved for
 * theta = (<f, c^2> - rho u^2) / (D rho). */
double ora_node_theta(const double *f, double rho, double ux, double uy) {
    double c2f = 0.0;
    for (int i = 0; i < ORA_Q; ++i)
        c2f += (double)(ORA_C[i][0] * ORA_C[i][0] + ORA_C[i][1] * ORA_C[i][1]) * f[i];
    return (c2f - rho * (ux * ux + uy * uy)) / ((double)ORA_D * rho);
}

/* One node's collision.  OReg (Eq. 7): post_i = f_i^eq + (1 - 1/tau) f_i^OReg.
 * BGK (Eq. 1): post_i = f_i - (1/tau) (f_i - f_i^eq).  With theta_local the
 * guided equilibrium and Eq. 6 take the node's own temperature. */
void ora_collide_node(const ora_params *p, const double *f, double *post) {
    double rho, ux, uy, feq[ORA_Q];
    ora_node_moments(f, &rho, &ux, &uy);
    const double theta = p->theta_local ? ora_node_theta(f, rho, ux, uy) : p->theta;
    ora_feq(p->eq, theta, rho, ux, uy, feq);
    if (p->coll == 0) {
        double foreg[ORA_Q];
        ora_foreg(f, feq, rho, ux, uy, ora_theta_eff(p->eq, theta), foreg);
        for (int i = 0; i < ORA_Q; ++i)
            post[i] = feq[i] + (1.0 - 1.0 / p->tau) * foreg[i];
    } else {
        for (int i = 0; i < ORA_Q; ++i)
            post[i] = f[i] - (1.0 / p->tau) * (f[i] - feq[i]);
    }
}

/* Full-way bounce-back at a solid wall node (Sec. IV shock tube): the node
 * does not collide; each population arriving along c_i leaves along -c_i,
 * post_i = f_k with c_k = -c_i. */
void ora_bounce_back_node(const double *f, double *post) {
    for (int i = 0; i < ORA_Q; ++i) {
        for (int k = 0; k < ORA_Q; ++k) {
            if (ORA_C[k][0] == -ORA_C[i][0] && ORA_C[k][1] == -ORA_C[i][1]) post[i] = f[k];
        }
    }
}

static int64_t ora_wrap(int64_t v, int64_t n) {
    int64_t r = v % n;
    return r < 0 ? r + n : r;
}

/* Streaming of Eqs. 1 and 7: the value leaving x in direction i arrives at
 * x + c_i; both axes are periodic.  dst must not alias post. */
void ora_stream(int32_t nx, int32_t ny, const double *post, double *dst) {
    const int64_t N = (int64_t)nx * ny;
    for (int i = 0; i < ORA_Q; ++i) {
        for (int64_t y = 0; y < ny; ++y) {
            const int64_t yd = ora_wrap(y + ORA_C[i][1], ny);
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t xd = ora_wrap(x + ORA_C[i][0], nx);
                dst[i * N + yd * nx + xd] = post[i * N + y * nx + x];
            }
        }
    }
}

/* One time step S_t -> S_{t+1}: collide at every node (bounce back at wall
 * nodes), then push each post-collision population to its neighbour; the
 * push wraps periodically in both axes (with walls, what crosses between the
 * two wall columns stays inside the walls).  src and dst must not alias.
 * Rows are independent, so they may run on several host threads without
 * changing any result. */
void ora_step(const ora_params *p, const double *src, double *dst) {
    const int64_t nx = p->nx, ny = p->ny, N = nx * ny;
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < ny; ++y) {
        for (int64_t x = 0; x < nx; ++x) {
            double f[ORA_Q], post[ORA_Q];
            for (int i = 0; i < ORA_Q; ++i) f[i] = src[i * N + y * nx + x];
            if (p->walls && (x == 0 || x == nx - 1))
                ora_bounce_back_node(f, post);
            else
                ora_collide_node(p, f, post);
            for (int i = 0; i < ORA_Q; ++i) {
                const int64_t yd = ora_wrap(y + ORA_C[i][1], ny);
                const int64_t xd = ora_wrap(x + ORA_C[i][0], nx);
                dst[i * N + yd * nx + xd] = post[i];
            }
        }
    }
}

/* Runs nsteps steps.  f holds S_t on entry and S_{t+nsteps} on return;
 * work is a caller buffer of the same size. */
void ora_run(const ora_params *p, double *f, double *work, int64_t nsteps) {
    const int64_t n = (int64_t)ORA_Q * p->nx * p->ny;
    double *a = f, *b = work;
    for (int64_t s = 0; s < nsteps; ++s) {
        ora_step(p, a, b);
        double *t = a; a = b; b = t;
    }
    if (a != f)
        for (int64_t j = 0; j < n; ++j) f[j] = a[j];
}

/* S_0 = f^eq(rho(x), u(x)) at every node (zero non-equilibrium start). */
void ora_init_equilibrium(const ora_params *p, const double *rho, const double *ux,
                          const double *uy, double *f) {
    const int64_t N = (int64_t)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double feq[ORA_Q];
        ora_feq(p->eq, p->theta, rho[n], ux[n], uy[n], feq);
        for (int i = 0; i < ORA_Q; ++i) f[i * N + n] = feq[i];
    }
}

/* Eq. 5: the Navier-Stokes-level populations of Eq. 4 projected on the
 * lattice,
 *   f_i^(1) = -tau f_i^eq sum_{a,b} (C_ia C_ib - C_i^2 delta_ab / D)
 *                                  * (d_b u_a + d_a u_b) / (2 theta),
 * with C_i = c_i - u and the velocity gradient grad[a][b] = d_b u_a of one
 * node.  theta_eff is the temperature of Eq. 6 (ora_theta_eff). */
void ora_first_order(double tau, double theta_eff, const double *feq, double ux, double uy,
                     const double *grad /* [2][2] */, double *f1 /* [9] */) {
    const double u[ORA_D] = {ux, uy};
    for (int i = 0; i < ORA_Q; ++i) {
        double Cp[ORA_D]; /* peculiar velocity C_i */
        for (int a = 0; a < ORA_D; ++a) Cp[a] = (double)ORA_C[i][a] - u[a];
        const double Cp2 = Cp[0] * Cp[0] + Cp[1] * Cp[1];
        double contraction = 0.0;
        for (int a = 0; a < ORA_D; ++a) {
            for (int b = 0; b < ORA_D; ++b) {
                const double delta = (a == b) ? 1.0 : 0.0;
                const double rate = (grad[a * ORA_D + b] + grad[b * ORA_D + a]) / (2.0 * theta_eff);
                contraction += (Cp[a] * Cp[b] - Cp2 * delta / (double)ORA_D) * rate;
            }
        }
        f1[i] = -tau * feq[i] * contraction;
    }
}

/* S_0 = f^eq + f^(1) (Eq. 5) at every node, from the density, velocity and
 * velocity-gradient fields; grad holds d_b u_a at grad[(a*2 + b)*N + n]. */
void ora_init_first_order(const ora_params *p, const double *rho, const double *ux,
                          const double *uy, const double *grad, double *f) {
    const int64_t N = (int64_t)p->nx * p->ny;
    const double theta_eff = ora_theta_eff(p->eq, p->theta);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double feq[ORA_Q], f1[ORA_Q], g[ORA_D * ORA_D];
        for (int ab = 0; ab < ORA_D * ORA_D; ++ab) g[ab] = grad[ab * N + n];
        ora_feq(p->eq, p->theta, rho[n], ux[n], uy[n], feq);
        ora_first_order(p->tau, theta_eff, feq, ux[n], uy[n], g, f1);
        for (int i = 0; i < ORA_Q; ++i) f[i * N + n] = feq[i] + f1[i];
    }
}

/* Macroscopic fields of S_t: rho, u and the local temperature
 * theta_loc = (<f, c^2> - rho u^2) / (D rho), from E = (D p + rho u^2)/2 and
 * p = rho theta (Eq. 2a and the definitions after Eq. 2). */
void ora_fields(int32_t nx, int32_t ny, const double *f, double *rho, double *ux,
                double *uy, double *theta_loc) {
    const int64_t N = (int64_t)nx * ny;
    for (int64_t n = 0; n < N; ++n) {
        double r = 0.0, jx = 0.0, jy = 0.0, c2f = 0.0;
        for (int i = 0; i < ORA_Q; ++i) {
            const double fi = f[i * N + n];
            r += fi;
            jx += (double)ORA_C[i][0] * fi;
            jy += (double)ORA_C[i][1] * fi;
            c2f += (double)(ORA_C[i][0] * ORA_C[i][0] + ORA_C[i][1] * ORA_C[i][1]) * fi;
        }
        rho[n] = r;
        ux[n] = jx / r;
        uy[n] = jy / r;
        if (theta_loc) {
            const double u2 = ux[n] * ux[n] + uy[n] * uy[n];
            theta_loc[n] = (c2f - r * u2) / ((double)ORA_D * r);
        }
    }
}
