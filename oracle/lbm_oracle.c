/*
 * Plain FP64 CPU oracle for the D2Q9 BGK lattice Boltzmann solver.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into the oracle's own shared
 * library and is called only by the tests, by __graft_entry__.smoke() and by the
 * CPU-baseline legs of bench.py.  It shares no code with the CUDA library and is
 * written to be checked against the paper by eye, not to be fast.
 *
 * What it follows (arXiv 2508.13867):
 *   - Sec. 3, lattice Boltzmann equation and its collide/stream split;
 *   - Eq. bgkCollision (BGK collision with relaxation time tau > 1/2);
 *   - Eq. equilibrium (second-order equilibrium, full rho-weighted form);
 *   - the moment definitions rho = sum f_i, rho u = sum c_i f_i;
 *   - the D2Q9 velocity set and Eq. weightsDdQ9 (4/9, 1/9, 1/36), c_s^2 = 1/3;
 *   - Sec. 8.2, Taylor-Green vortex: periodic in both directions, tau = nu/c_s^2 + 1/2,
 *     discrete kinetic energy K(t) = 2/(nx ny u0^2) sum (u^2 + v^2);
 *   - Sec. 8.1, flow past a cylinder: parabolic inflow 4 u y (H - y)/H^2, no-slip walls,
 *     drag/lift coefficients C = 2F/(rho u^2 D), equilibrium initialisation, inflow ramp.
 *
 * Readings taken where the paper is silent (each is listed in the design notes):
 *   - D2Q9 order c = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1);
 *   - TGV phase u = U0 sin(kx)cos(ky), v = -U0 cos(kx)sin(ky), pressure
 *     p = U0^2/4 (cos 2kx + cos 2ky), density rho = 1 + 3p, populations start at
 *     equilibrium; optional extra divergence-free modes m = 2, 3 of amplitude A_m;
 *   - channel: halfway bounce-back on walls (y = 0 and y = ny faces) and on a
 *     staircase obstacle mask; the inlet is a moving-wall bounce-back at the x = 0
 *     face with the parabolic profile at the link midpoint (peak 1.5 x mean);
 *     the outlet is a pressure condition: anti-bounce-back at the x = nx face with
 *     rho_w = 1 and the wall velocity taken from the outlet node itself (zero
 *     gradient); forces by momentum exchange on obstacle links;
 *     ramp 1/2 (1 - cos(pi t / T_r)) for t < T_r;
 *   - obstacle scheme, selectable: halfway bounce-back on the staircase, or the
 *     linear interpolated bounce-back of Bouzidi, Firdaouss and Lallemand (2001),
 *     which Sec. 8.1 names for the cylinder surface.  For a link from fluid node x
 *     along c_k into the obstacle, q is the fraction of the link at which it meets
 *     the circle, and the population returning to x is
 *         q <  1/2:  f_kbar(x, t+1) = 2q f*_k(x, t) + (1 - 2q) f_k(x, t+1),
 *         q >= 1/2:  f_kbar(x, t+1) = f*_k(x, t) / (2q) + (1 - 1/(2q)) f*_kbar(x, t),
 *     where f_k(x, t+1) is the population streamed into x along c_k by the other
 *     rules (f*_k(x - c_k, t) for the fluid node upstream); the force is the momentum
 *     exchanged on the links, F = sum c_k (f*_k(x, t) + f_kbar(x, t+1)), taken after
 *     the stream (for halfway bounce-back this is 2 sum c_k f*_k(x, t)).
 *   - inlet/outlet scheme, selectable: the moving-wall and anti-bounce-back rules above at
 *     the end faces, or interpolated conditions on the end columns, the finite-difference
 *     velocity-gradient scheme that Latt et al. (2008) describe and Sec. 8.1 cites: after the
 *     stream, every population of a node of column 0 (inlet) or nx - 1 (outlet) is replaced by
 *     f_i = f_i^eq(rho, u) - 3 w_i rho tau Q_i:S, Q_i = c_i c_i - I/3, S the strain rate from
 *     finite differences (second-order one-sided across the column, central along it, one-sided
 *     at its ends); inlet: u = (parabola at the node centre, 0), rho from the known populations
 *     by mass balance, rho = (f_0 + f_2 + f_4 + 2 (f_3 + f_6 + f_7)) / (1 - u_x); outlet:
 *     rho = 1, u_x = (f_0 + f_2 + f_4 + 2 (f_1 + f_5 + f_8)) / rho - 1, u_y that of the node
 *     beside it (zero normal gradient).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double WGT[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

enum { ORACLE_TGV = 0, ORACLE_CHANNEL = 1, ORACLE_TGV_PERTURBED = 2 };

/* One deterministic run (one sample).  All lengths are in lattice units. */
typedef struct {
    int32_t kind;        /* ORACLE_TGV or ORACLE_CHANNEL */
    int32_t nx, ny;      /* lattice size */
    int64_t steps;       /* number of time steps (TGV) or step cap (channel) */
    double nu;           /* lattice kinematic viscosity, tau = 3 nu + 1/2 */
    double u0;           /* TGV amplitude, or channel mean inflow velocity */
    double amp2, amp3;   /* TGV: absolute amplitudes of the k2 = 2k and k3 = 3k modes */
    double u_ref;        /* TGV: normaliser of K(t); channel: unused */
    double cyl_cx, cyl_cy, cyl_r; /* channel: obstacle circle (r <= 0: no obstacle) */
    int64_t ramp_steps;  /* channel: inflow ramp length T_r (0: no ramp) */
    int64_t qoi_every;   /* stride of the QoI series (0: no series) */
    double steady_tol;   /* channel: stop when |dC_D|/|C_D| < tol between checks (0: never) */
    double pert[4];      /* perturbed TGV: zeta_00, zeta_01, zeta_10, zeta_11 (lattice velocity units) */
    int32_t obstacle_bc; /* channel obstacle: 0 halfway bounce-back, 1 Bouzidi linear interpolation */
    int32_t inout_bc;    /* channel inlet/outlet: 0 moving-wall / anti-bounce-back at the end faces,
                            1 interpolated (finite-difference) conditions on the end columns */
} oracle_case;

/* Per-run outputs.  Arrays are row-major [ny][nx]; any pointer may be NULL. */
typedef struct {
    double *u, *v, *rho;   /* final macroscopic fields (zero on obstacle nodes) */
    double *series;        /* QoI series: K(t) (TGV) or C_D(t) (channel) at t = 0, e, 2e, ... */
    double *series_cl;     /* channel only: C_L(t) at the same times */
    int64_t series_len;    /* capacity of series / series_cl */
    double scalars[8];     /* [0] K(T), [1] mass, [2] x-momentum, [3] y-momentum,
                              [4] C_D, [5] C_L, [6] steps run, [7] unused */
} oracle_out;

static double feq(int i, double rho, double ux, double uy) {
    /* Eq. equilibrium with c_s^2 = 1/3. */
    double cu = CX[i] * ux + CY[i] * uy;
    double uu = ux * ux + uy * uy;
    return WGT[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

static void moments(const double *f, int64_t plane, int64_t n, double *rho, double *ux,
                    double *uy) {
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < Q; ++i) {
        double fi = f[i * plane + n];
        r += fi;
        jx += CX[i] * fi;
        jy += CY[i] * fi;
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
}

/* Staircase obstacle: node (x, y) with centre (x + 1/2, y + 1/2) strictly inside the circle. */
static int node_solid(const oracle_case *c, int x, int y) {
    if (c->kind != ORACLE_CHANNEL || c->cyl_r <= 0.0) return 0;
    double dx = (x + 0.5) - c->cyl_cx, dy = (y + 0.5) - c->cyl_cy;
    return dx * dx + dy * dy < c->cyl_r * c->cyl_r;
}

/* Fraction q of the link from node (x, y) along c_i at which it enters the obstacle circle:
 * the smaller root s of |P + s c_i - C|^2 = r^2, P = (x + 1/2, y + 1/2), C the centre. */
static double link_fraction(const oracle_case *c, int x, int y, int i) {
    double px = (x + 0.5) - c->cyl_cx, py = (y + 0.5) - c->cyl_cy;
    double a = (double)(CX[i] * CX[i] + CY[i] * CY[i]);
    double b = 2.0 * (CX[i] * px + CY[i] * py);
    double cc = px * px + py * py - c->cyl_r * c->cyl_r;
    return (-b - sqrt(b * b - 4.0 * a * cc)) / (2.0 * a);
}

/* Interpolated inlet (column 0) and outlet (column nx - 1) at the state of time tn, applied to
 * the post-stream populations f: velocities of the columns next to each boundary from their
 * moments, the boundary velocity and density as described in the header, the strain rate by
 * finite differences, then f = f^eq + f^neq on both boundary columns. */
static void interpolated_inout(const oracle_case *c, double *f, int64_t plane, double tau, int64_t tn);

/* Parabolic inflow profile evaluated at height yy (walls at 0 and H = ny), peak 1.5 x mean. */
static double inflow_u(const oracle_case *c, double yy, int64_t t) {
    double H = (double)c->ny;
    double umax = 1.5 * c->u0;
    double ramp = 1.0;
    if (c->ramp_steps > 0 && t < c->ramp_steps)
        ramp = 0.5 * (1.0 - cos(M_PI * (double)t / (double)c->ramp_steps));
    return 4.0 * umax * ramp * yy * (H - yy) / (H * H);
}

static void tgv_initial(const oracle_case *c, int x, int y, double *rho, double *ux,
                        double *uy) {
    double kx = 2.0 * M_PI / c->nx, ky = 2.0 * M_PI / c->ny;
    double U0 = c->u0;
    double u = U0 * sin(kx * x) * cos(ky * y);
    double v = -U0 * cos(kx * x) * sin(ky * y);
    u += c->amp2 * sin(2.0 * kx * x) * cos(2.0 * ky * y);
    v -= c->amp2 * cos(2.0 * kx * x) * sin(2.0 * ky * y);
    u += c->amp3 * sin(3.0 * kx * x) * cos(3.0 * ky * y);
    v -= c->amp3 * cos(3.0 * kx * x) * sin(3.0 * ky * y);
    double p = 0.25 * U0 * U0 * (cos(2.0 * kx * x) + cos(2.0 * ky * y));
    *rho = 1.0 + 3.0 * p;
    *ux = u;
    *uy = v;
}

/* Sec. 8.3 Taylor-Green vortex with four-dimensional uncertain initial velocity, on the periodic
 * square [0, 2 pi)^2 resolved by nx x ny nodes x = 2 pi i / nx:
 *   u = -U cos(2x) sin(2y), v = U sin(2x) cos(2y), U = u0 + eps(x, y),
 *   eps = 1/4 sum_{i,j in {0,1}} zeta_ij k_i(4x) k_j(4y), k_0 = sin, k_1 = cos,
 *   p = -U^2/4 (cos 4x + cos 4y) (the printed factor (2/2)^2 is 1), rho = 1 + 3 p. */
static void tgv_perturbed_initial(const oracle_case *c, int ix, int iy, double *rho, double *ux,
                                  double *uy) {
    double x = 2.0 * M_PI * ix / c->nx, y = 2.0 * M_PI * iy / c->ny;
    double kx[2] = {sin(4.0 * x), cos(4.0 * x)};
    double ky[2] = {sin(4.0 * y), cos(4.0 * y)};
    double eps = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) eps += c->pert[2 * i + j] * kx[i] * ky[j];
    double U = c->u0 + 0.25 * eps;
    *ux = -U * cos(2.0 * x) * sin(2.0 * y);
    *uy = U * sin(2.0 * x) * cos(2.0 * y);
    double p = -0.25 * U * U * (cos(4.0 * x) + cos(4.0 * y));
    *rho = 1.0 + 3.0 * p;
}

/* QoI of the current (post-stream) state: K(t) for the TGV. */
static double kinetic_energy(const oracle_case *c, const double *f, const unsigned char *solid) {
    int64_t plane = (int64_t)c->nx * c->ny;
    double s = 0.0;
    for (int64_t n = 0; n < plane; ++n) {
        if (solid[n]) continue;
        double rho, ux, uy;
        moments(f, plane, n, &rho, &ux, &uy);
        s += ux * ux + uy * uy;
    }
    return 2.0 * s / ((double)c->nx * (double)c->ny * c->u_ref * c->u_ref);
}

/* Run one sample.  Returns 0 on success, -1 on bad arguments, -2 on allocation failure. */
int oracle_run(const oracle_case *c, oracle_out *o) {
    if (!c || !o || c->nx < 2 || c->ny < 2 || c->steps < 0 || c->nu <= 0.0) return -1;
    if (c->kind == ORACLE_CHANNEL && c->inout_bc == 1 && (c->nx < 6 || c->ny < 3)) return -1;
    const int nx = c->nx, ny = c->ny;
    const int64_t plane = (int64_t)nx * ny;
    const double tau = 3.0 * c->nu + 0.5;
    const double omega = 1.0 / tau;

    double *f = (double *)malloc(sizeof(double) * Q * plane);
    double *fpost = (double *)malloc(sizeof(double) * Q * plane);
    unsigned char *solid = (unsigned char *)calloc((size_t)plane, 1);
    double *uout = (double *)calloc((size_t)2 * ny, sizeof(double)); /* outlet node velocity */
    if (!f || !fpost || !solid || !uout) {
        free(f);
        free(fpost);
        free(solid);
        free(uout);
        return -2;
    }
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) solid[(int64_t)y * nx + x] = (unsigned char)node_solid(c, x, y);

    /* Initial state: equilibrium populations of the initial macroscopic field. */
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int64_t n = (int64_t)y * nx + x;
            double rho = 1.0, ux = 0.0, uy = 0.0;
            if (c->kind == ORACLE_TGV) tgv_initial(c, x, y, &rho, &ux, &uy);
            if (c->kind == ORACLE_TGV_PERTURBED) tgv_perturbed_initial(c, x, y, &rho, &ux, &uy);
            if (solid[n]) ux = uy = 0.0;
            for (int i = 0; i < Q; ++i) f[i * plane + n] = feq(i, rho, ux, uy);
        }
    }

    const int bouzidi = c->kind == ORACLE_CHANNEL && c->cyl_r > 0.0 && c->obstacle_bc == 1;
    const double Dlat = 2.0 * c->cyl_r;
    const double force_norm = (c->kind == ORACLE_CHANNEL && Dlat > 0.0)
                                  ? 2.0 / (1.0 * c->u0 * c->u0 * Dlat)
                                  : 0.0;
    int64_t nseries = 0;
    double cd = 0.0, cl = 0.0, cd_prev = NAN;
    if (o->series && o->series_len > 0 && c->qoi_every > 0 && c->kind != ORACLE_CHANNEL)
        o->series[nseries++] = kinetic_energy(c, f, solid);

    int64_t t;
    for (t = 0; t < c->steps; ++t) {
        /* Collision (Eq. bgkCollision) on every fluid node. */
        double fx = 0.0, fy = 0.0;
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                int64_t n = (int64_t)y * nx + x;
                if (solid[n]) continue;
                double rho, ux, uy;
                moments(f, plane, n, &rho, &ux, &uy);
                for (int i = 0; i < Q; ++i) {
                    double fi = f[i * plane + n];
                    fpost[i * plane + n] = fi - omega * (fi - feq(i, rho, ux, uy));
                }
                if (x == nx - 1) {
                    uout[2 * y] = ux;
                    uout[2 * y + 1] = uy;
                }
                /* Momentum exchange on links into the obstacle (halfway bounce-back). */
                if (c->kind == ORACLE_CHANNEL && !bouzidi) {
                    for (int i = 1; i < Q; ++i) {
                        int xn = x + CX[i], yn = y + CY[i];
                        if (xn < 0 || xn >= nx || yn < 0 || yn >= ny) continue;
                        if (solid[(int64_t)yn * nx + xn]) {
                            fx += 2.0 * CX[i] * fpost[i * plane + n];
                            fy += 2.0 * CY[i] * fpost[i * plane + n];
                        }
                    }
                }
            }
        }
        /* Streaming f_i(x + c_i, t + 1) = f*_i(x, t), written in pull form with the boundary rules. */
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                int64_t n = (int64_t)y * nx + x;
                if (solid[n]) continue;
                for (int i = 0; i < Q; ++i) {
                    int sx = x - CX[i], sy = y - CY[i];
                    double val;
                    if (c->kind != ORACLE_CHANNEL) {
                        sx = (sx + nx) % nx;
                        sy = (sy + ny) % ny;
                        val = fpost[i * plane + (int64_t)sy * nx + sx];
                    } else if (sy < 0 || sy >= ny) {
                        val = fpost[OPP[i] * plane + n]; /* wall: halfway bounce-back */
                    } else if (sx < 0) {
                        /* inlet: moving-wall bounce-back, wall velocity at the link midpoint */
                        double uw = inflow_u(c, (y + 0.5) - 0.5 * CY[i], t);
                        val = fpost[OPP[i] * plane + n] + 6.0 * WGT[i] * CX[i] * uw;
                    } else if (sx >= nx) {
                        /* outlet: anti-bounce-back, rho_w = 1, u_w = velocity of this node at t */
                        double ux = uout[2 * y], uy = uout[2 * y + 1];
                        double cu = CX[i] * ux + CY[i] * uy;
                        val = -fpost[OPP[i] * plane + n] +
                              2.0 * WGT[i] * 1.0 * (1.0 + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy));
                    } else if (solid[(int64_t)sy * nx + sx]) {
                        val = fpost[OPP[i] * plane + n]; /* obstacle: halfway bounce-back */
                    } else {
                        val = fpost[i * plane + (int64_t)sy * nx + sx];
                    }
                    f[i * plane + n] = val;
                }
            }
        }
        if (bouzidi) {
            /* Interpolated bounce-back on the obstacle links (the pull above left the halfway
             * value there), then the momentum exchanged on them. */
            for (int y = 0; y < ny; ++y) {
                for (int x = 0; x < nx; ++x) {
                    int64_t n = (int64_t)y * nx + x;
                    if (solid[n]) continue;
                    for (int k = 1; k < Q; ++k) {
                        int xn = x + CX[k], yn = y + CY[k];
                        if (xn < 0 || xn >= nx || yn < 0 || yn >= ny || !solid[(int64_t)yn * nx + xn]) continue;
                        int kb = OPP[k];
                        double q = link_fraction(c, x, y, k);
                        double back;
                        if (q < 0.5)
                            back = 2.0 * q * fpost[k * plane + n] + (1.0 - 2.0 * q) * f[k * plane + n];
                        else
                            back = fpost[k * plane + n] / (2.0 * q) + (1.0 - 1.0 / (2.0 * q)) * fpost[kb * plane + n];
                        f[kb * plane + n] = back;
                        fx += CX[k] * (fpost[k * plane + n] + back);
                        fy += CY[k] * (fpost[k * plane + n] + back);
                    }
                }
            }
        }
        if (c->kind == ORACLE_CHANNEL && c->inout_bc == 1) interpolated_inout(c, f, plane, tau, t + 1);
        if (c->kind == ORACLE_CHANNEL) {
            cd = fx * force_norm;
            cl = fy * force_norm;
        }
        int64_t tn = t + 1; /* time of the state now held in f */
        if (c->qoi_every > 0 && tn % c->qoi_every == 0) {
            if (c->kind != ORACLE_CHANNEL) {
                if (o->series && nseries < o->series_len)
                    o->series[nseries++] = kinetic_energy(c, f, solid);
            } else {
                if (o->series && nseries < o->series_len) {
                    o->series[nseries] = cd;
                    if (o->series_cl) o->series_cl[nseries] = cl;
                    nseries++;
                }
                if (c->steady_tol > 0.0) {
                    int done = !isnan(cd_prev) && fabs(cd - cd_prev) < c->steady_tol * fabs(cd);
                    cd_prev = cd;
                    if (done) {
                        ++t;
                        break;
                    }
                }
            }
        }
    }

    double mass = 0.0, mx = 0.0, my = 0.0;
    for (int64_t n = 0; n < plane; ++n) {
        double rho = 0.0, ux = 0.0, uy = 0.0;
        if (!solid[n]) {
            moments(f, plane, n, &rho, &ux, &uy);
            mass += rho;
            mx += rho * ux;
            my += rho * uy;
        }
        if (o->u) o->u[n] = ux;
        if (o->v) o->v[n] = uy;
        if (o->rho) o->rho[n] = rho;
    }
    o->scalars[0] = c->u_ref > 0.0 ? kinetic_energy(c, f, solid) : 0.0;
    o->scalars[1] = mass;
    o->scalars[2] = mx;
    o->scalars[3] = my;
    o->scalars[4] = cd;
    o->scalars[5] = cl;
    o->scalars[6] = (double)t;
    o->scalars[7] = 0.0;

    free(f);
    free(fpost);
    free(solid);
    free(uout);
    return 0;
}

static void interpolated_inout(const oracle_case *c, double *f, int64_t plane, double tau, int64_t tn) {
    const int nx = c->nx, ny = c->ny;
    /* velocity (ux, uy) and density of the columns 0, 1, 2 (inlet side) and nx - 3, nx - 2,
     * nx - 1 (outlet side), indexed [side][k][y], k = distance from the boundary column */
    double *ux = (double *)malloc(sizeof(double) * 6 * ny);
    double *uy = (double *)malloc(sizeof(double) * 6 * ny);
    double *rb = (double *)malloc(sizeof(double) * 2 * ny);
    if (!ux || !uy || !rb) {
        free(ux);
        free(uy);
        free(rb);
        return;
    }
#define U_AT(a, side, k, y) a[((side) * 3 + (k)) * ny + (y)]
    for (int side = 0; side < 2; ++side) {
        for (int k = 1; k < 3; ++k) {
            const int x = side == 0 ? k : nx - 1 - k;
            for (int y = 0; y < ny; ++y) {
                double r, vx, vy;
                moments(f, plane, (int64_t)y * nx + x, &r, &vx, &vy);
                U_AT(ux, side, k, y) = vx;
                U_AT(uy, side, k, y) = vy;
            }
        }
    }
    for (int y = 0; y < ny; ++y) {
        const int64_t ni = (int64_t)y * nx, no = (int64_t)y * nx + nx - 1;
        const double uin = inflow_u(c, y + 0.5, tn);
        U_AT(ux, 0, 0, y) = uin;
        U_AT(uy, 0, 0, y) = 0.0;
        rb[y] = (f[0 * plane + ni] + f[2 * plane + ni] + f[4 * plane + ni] +
                 2.0 * (f[3 * plane + ni] + f[6 * plane + ni] + f[7 * plane + ni])) /
                (1.0 - uin);
        rb[ny + y] = 1.0;
        U_AT(ux, 1, 0, y) = (f[0 * plane + no] + f[2 * plane + no] + f[4 * plane + no] +
                             2.0 * (f[1 * plane + no] + f[5 * plane + no] + f[8 * plane + no])) /
                                rb[ny + y] -
                            1.0;
        U_AT(uy, 1, 0, y) = U_AT(uy, 1, 1, y);
    }
    for (int side = 0; side < 2; ++side) {
        const int x = side == 0 ? 0 : nx - 1;
        const double sgn = side == 0 ? 1.0 : -1.0; /* the column index k grows along +x (inlet) or -x */
        for (int y = 0; y < ny; ++y) {
            double dxu, dxv, dyu, dyv;
            /* d/dx: second-order one-sided from the boundary column inwards */
            dxu = sgn * (-3.0 * U_AT(ux, side, 0, y) + 4.0 * U_AT(ux, side, 1, y) - U_AT(ux, side, 2, y)) / 2.0;
            dxv = sgn * (-3.0 * U_AT(uy, side, 0, y) + 4.0 * U_AT(uy, side, 1, y) - U_AT(uy, side, 2, y)) / 2.0;
            /* d/dy along the boundary column: central, one-sided at its ends */
            if (y == 0) {
                dyu = (-3.0 * U_AT(ux, side, 0, 0) + 4.0 * U_AT(ux, side, 0, 1) - U_AT(ux, side, 0, 2)) / 2.0;
                dyv = (-3.0 * U_AT(uy, side, 0, 0) + 4.0 * U_AT(uy, side, 0, 1) - U_AT(uy, side, 0, 2)) / 2.0;
            } else if (y == ny - 1) {
                dyu = (3.0 * U_AT(ux, side, 0, y) - 4.0 * U_AT(ux, side, 0, y - 1) + U_AT(ux, side, 0, y - 2)) / 2.0;
                dyv = (3.0 * U_AT(uy, side, 0, y) - 4.0 * U_AT(uy, side, 0, y - 1) + U_AT(uy, side, 0, y - 2)) / 2.0;
            } else {
                dyu = (U_AT(ux, side, 0, y + 1) - U_AT(ux, side, 0, y - 1)) / 2.0;
                dyv = (U_AT(uy, side, 0, y + 1) - U_AT(uy, side, 0, y - 1)) / 2.0;
            }
            const double sxx = dxu, syy = dyv, sxy = 0.5 * (dyu + dxv);
            const double rho = rb[side * ny + y], vx = U_AT(ux, side, 0, y), vy = U_AT(uy, side, 0, y);
            const int64_t n = (int64_t)y * nx + x;
            for (int i = 0; i < Q; ++i) {
                const double q = (CX[i] * CX[i] - 1.0 / 3.0) * sxx + (CY[i] * CY[i] - 1.0 / 3.0) * syy +
                                 2.0 * CX[i] * CY[i] * sxy;
                f[i * plane + n] = feq(i, rho, vx, vy) - 3.0 * WGT[i] * rho * tau * q;
            }
        }
    }
#undef U_AT
    free(ux);
    free(uy);
    free(rb);
}

/* Run a batch of independent samples, one sample per OpenMP thread (sample-level parallelism). */
int oracle_run_batch(const oracle_case *cases, oracle_out *outs, int64_t n, int threads) {
    int rc = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(min : rc)
#endif
    for (int64_t s = 0; s < n; ++s) {
        int r = oracle_run(&cases[s], &outs[s]);
        if (r < rc) rc = r;
    }
    return rc;
}

/* Obstacle mask exactly as the oracle uses it, row-major [ny][nx], 1 = solid. */
int oracle_obstacle_mask(const oracle_case *c, unsigned char *mask) {
    if (!c || !mask) return -1;
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) mask[(int64_t)y * c->nx + x] = (unsigned char)node_solid(c, x, y);
    return 0;
}

/* Link fraction q of the link from fluid node (x, y) along direction i (test access). */
double oracle_link_fraction(const oracle_case *c, int x, int y, int i) {
    if (!c || i < 1 || i >= Q) return NAN;
    return link_fraction(c, x, y, i);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
