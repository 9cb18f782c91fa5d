/*
 * lbmdem_oracle.c -- plain, slow FP64 CPU reference of the coupled LBM-DEM
 * time step of Cheng, Luding, Rivas, Harting, Magnanimo, "Hydro-
 * micromechanical modeling of wave propagation in saturated granular media"
 * (arXiv 1808.08921).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test suite, the package smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header or
 * table with the CUDA implementation.
 *
 * What it computes, in the paper's order (one call of orc_step):
 *   1. paint the solid map from the particle positions (Section 2.3), by
 *      brute force over every particle and every periodic image, and apply
 *      the node-conversion momentum corrections (Eqs. 16, 17);
 *   2. BGK collision on every fluid node (Eqs. 4, 6, 7, 8);
 *   3. streaming (Eq. 5) with half-way moving-wall bounce-back on every
 *      fluid-solid link (Eq. 14) and the link force and torque (Eqs. 15,
 *      18, 19), on a second lattice (two-lattice push scheme).  The link
 *      momentum is counted about the rest state, c_d (f~_d + f_d* - 2 w_d
 *      rho_f): the mean fluid pressure acts on the whole grain surface (the
 *      paper's granular stress, Eq. 13, is an effective stress, and its
 *      confining pressures of 0.1-30 MPa are set by the overlaps while the
 *      mean lattice pressure maps to 2.25 GPa, Table 1).  A fully wetted
 *      sphere is unaffected; on touching spheres the mean pressure would
 *      otherwise press on the unwetted contact caps;
 *   4. the pressure inlet with the oscillating density (Section 2.4,
 *      Zou-He form for D3Q19, Eq. 25 and Table 2) and the outlet;
 *   5. K velocity-Verlet DEM substeps with Hertz normal and incremental
 *      Mindlin tangential contacts capped by Coulomb friction (Eqs. 9-12),
 *      the hydrodynamic force and torque held fixed over the K substeps.
 *      The force and torque that drive the sphere in step t are the mean of
 *      the sums of Eqs. 18-19 of steps t and t-1 (zero before the first
 *      step): the half-way bounce-back force alternates from step to step
 *      (Ladd's momentum-exchange method, cited in Section 2.3, averages it
 *      over two steps), and applied raw it drives the fluid pockets at the
 *      contact necks of spheres with rho_p / rho_f ~ 2.5 unstable.
 *
 * Readings where the paper is silent or garbled (each is stated where it is
 * used): index order and opposites from the columns of Eq. 3; moving-wall
 * density rho_w = rho_f; conversion signs (particle gains the momentum of a
 * covered node, loses rho_bar * V_b for an uncovered node); boundary planes
 * x = 0 and x = nx-1 are never solid; owner of a node covered by several
 * spheres = smallest |x - X|^2 / R^2 (lowest index on a tie); populations arriving from outside the x
 * range start as the node's own reversed post-collision value (a resting
 * wall) before the inlet/outlet overwrite them; zero-gradient outlet copies
 * the unknown populations from the upstream node when that node is fluid.
 *
 * Threads (OpenMP, when compiled with it): the lattice loops run over
 * x-planes in parallel and the contact search over the lower-index sphere
 * of each pair.  Every floating-point sum has a fixed order whatever the
 * thread count: link forces and torques (Eqs. 18-19) are summed per
 * x-plane, then plane by plane in x order; pair contact forces are
 * evaluated in parallel and added to the spheres in the serial pair order.
 * One thread or many give bit-identical results.
 *
 * orc_set_link_form(s, 1) switches the link momentum to the literal Eq. 15,
 * c_d (f~_d + f_d*), so that the tests can pin the rest-state reading
 * against it (the two differ only by 2 w_d rho_f c_d summed over the links,
 * which vanishes over the closed staircase of a fully wetted sphere).
 *
 * orc_set_coupling(s, 1) replaces the momentum-exchange coupling by a
 * smooth surrogate for gradients in the sphere positions (outside the
 * paper's chosen method; the paper names the Noble-Torczynski
 * partially-saturated scheme as the alternative family, Section 1): every
 * node carries populations and collides with a solid-fraction-weighted
 * operator (psm_step below), the spheres stay fixed.
 *
 * Parity pins (tests/test_oracle_*.py): equilibrium moments, BGK
 * conservation, exact streaming shifts, Zou-He moment identities, mass
 * conservation with static spheres in a closed box, y/z momentum balance
 * with moving spheres in a periodic box, Hertz closed form, head-on
 * collision time and energy, Coulomb cap, multiple periodic images, the
 * damped plane wave of Eq. 27.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#include "lbmdem_oracle.h"

#define Q 19

/* D3Q19 velocities: the 19 columns of the matrix in Eq. 3, in order. */
static const int CX[Q] = {1, -1, 0, 0, 0, 0, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0};
static const int CZ[Q] = {0, 0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 1, -1, 0};
static double WT[Q]; /* Eq. 8: 1/3, 1/18, 1/36 by |c| */
static int OPP[Q];   /* d* with c_d* = -c_d (Section 2.3) */
static int tables_ready = 0;

static void init_tables(void) {
    if (tables_ready) return;
    for (int m = 0; m < Q; ++m) {
        int c2 = CX[m] * CX[m] + CY[m] * CY[m] + CZ[m] * CZ[m];
        WT[m] = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
        for (int k = 0; k < Q; ++k)
            if (CX[k] == -CX[m] && CY[k] == -CY[m] && CZ[k] == -CZ[m]) OPP[m] = k;
    }
    tables_ready = 1;
}

typedef struct {
    int j, sx, sy, sz; /* partner index and periodic image (in box lengths) */
    double ft[3];      /* tangential force on the lower-index particle */
} hist_t;

typedef struct {
    hist_t* e;
    int n, cap;
} hist_list;

/* one sphere's link force and torque summed over one x-plane */
typedef struct {
    int p;
    double F[3], T[3];
} plane_sum;

typedef struct {
    plane_sum* e;
    int n, cap;
} plane_list;

/* one pair contact found from the lower-index sphere i (Eqs. 11-12) */
typedef struct {
    int j;
    double F[3], ti[3], tj[3];
} pair_hit;

typedef struct {
    pair_hit* e;
    int n, cap;
} pair_list;

struct orc_sim {
    orc_params p;
    long N;
    int px; /* x periodic */
    double* f;
    double* fn;
    int* owner; /* -1 fluid, else the covering sphere of smallest |x - X|^2 / R^2 */
    int* owner_new;
    double* best; /* that ratio, per node, while painting */
    /* particles */
    int np;
    double *X, *V, *W, *q, *R, *m, *I;
    unsigned char* fixed;
    double *Fh, *Th, *Fc, *Tc;
    double *Fh_prev, *Th_prev; /* sums of Eqs. 18-19 of the previous step */
    double *Fa, *Ta;           /* applied: mean of this and the previous step */
    double *Vh, *Wh;
    hist_list* hist;
    /* source */
    int waveform;
    double amp, omega, t0;
    long long t_n;
    long long t;
    double* trace;
    long long trace_len, trace_cap;
    int have_packing;
    int link_literal;       /* 1: link momentum c_d (f~_d + f_d*) as printed in Eq. 15 */
    int psm;                /* 1: the smooth partially-saturated surrogate (orc_set_coupling) */
    double* eps;            /* its solid fraction per node, if given (orc_psm_set_fraction) */
    double* eps_auto;       /* else from the (fixed) spheres, computed once per packing */
    plane_list* plane_acc;  /* [nx] link sums of each x-plane */
    pair_list* pairs;       /* [np] contacts found from each lower-index sphere */
};

static inline long nidx(const orc_sim* s, int x, int y, int z) {
    return ((long)x * s->p.ny + y) * s->p.nz + z;
}

static inline int wrapi(int a, int L) {
    int r = a % L;
    return r < 0 ? r + L : r;
}

/* minimum-image component for a periodic axis */
static inline double minimg(double d, double L, int periodic) {
    if (!periodic) return d;
    return d - L * floor(d / L + 0.5);
}

static inline void cross(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ---------------------------------------------------------------- lattice */

void orc_lattice(int* cx, int* cy, int* cz, double* w, int* opp) {
    init_tables();
    for (int m = 0; m < Q; ++m) {
        cx[m] = CX[m];
        cy[m] = CY[m];
        cz[m] = CZ[m];
        w[m] = WT[m];
        opp[m] = OPP[m];
    }
}

/* Eq. 6 with c_s^2 = 1/3 (Section 2.1). */
void orc_equilibrium(double rho, double ux, double uy, double uz, double* feq) {
    init_tables();
    double uu = ux * ux + uy * uy + uz * uz;
    for (int m = 0; m < Q; ++m) {
        double cu = CX[m] * ux + CY[m] * uy + CZ[m] * uz;
        feq[m] = WT[m] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* Eq. 7 */
static void moments(const double* fm, double* rho, double* j) {
    double r = 0, jx = 0, jy = 0, jz = 0;
    for (int m = 0; m < Q; ++m) {
        r += fm[m];
        jx += fm[m] * CX[m];
        jy += fm[m] * CY[m];
        jz += fm[m] * CZ[m];
    }
    *rho = r;
    j[0] = jx;
    j[1] = jy;
    j[2] = jz;
}

/* Eq. 4: one node, in place. */
void orc_collide_node(double* fm, double tau) {
    init_tables();
    double rho, j[3], feq[Q];
    moments(fm, &rho, j);
    orc_equilibrium(rho, j[0] / rho, j[1] / rho, j[2] / rho, feq);
    for (int m = 0; m < Q; ++m) fm[m] = fm[m] + (feq[m] - fm[m]) / tau;
}

/* Section 2.4: D3Q19 pressure boundary on an x-normal face.  The unknown
 * populations are rebuilt from the known ones by bouncing back the
 * non-equilibrium part, with tangential velocity zero and transverse
 * momentum corrections N_y, N_z.  The printed z-normal form has two typos
 * (f5 from f3, and the sign of the rho*u/3 term in N); the x-normal form
 * below is the one that makes the moments come out exactly:
 *   inlet side (unknown c_x = +1), sgn = +1; outlet side (unknown c_x = -1),
 *   sgn = -1. */
void orc_pressure_face(double* fm, double rho_b, int side /* 0 inlet, 1 outlet */) {
    init_tables();
    /* 1-based paper indices -> 0-based: f1 -> fm[0] ... f19 -> fm[18] */
#define F(k) fm[(k) - 1]
    double rest = F(19) + F(3) + F(4) + F(5) + F(6) + F(15) + F(16) + F(17) + F(18);
    double Ny = 0.5 * (F(3) + F(15) + F(16) - F(4) - F(17) - F(18));
    double Nz = 0.5 * (F(5) + F(15) + F(17) - F(6) - F(16) - F(18));
    if (side == 0) {
        double rux = rho_b - (rest + 2.0 * (F(2) + F(11) + F(12) + F(13) + F(14)));
        F(1) = F(2) + rux / 3.0;
        F(7) = F(12) + rux / 6.0 - Ny;
        F(8) = F(11) + rux / 6.0 + Ny;
        F(9) = F(14) + rux / 6.0 - Nz;
        F(10) = F(13) + rux / 6.0 + Nz;
    } else {
        double rux = (rest + 2.0 * (F(1) + F(7) + F(8) + F(9) + F(10))) - rho_b;
        F(2) = F(1) - rux / 3.0;
        F(12) = F(7) - rux / 6.0 + Ny;
        F(11) = F(8) - rux / 6.0 - Ny;
        F(14) = F(9) - rux / 6.0 + Nz;
        F(13) = F(10) - rux / 6.0 - Nz;
    }
#undef F
}

/* Eq. 25 and Table 2: density imposed at the source at time t (steps done). */
double orc_source_density(const orc_sim* s, long long t) {
    double rf = s->p.rho_f;
    if (s->t_n >= 0 && t > s->t_n) return rf;
    double w = s->omega, tt = (double)t;
    switch (s->waveform) {
        case ORC_SINE: return rf + s->amp * sin(w * tt);
        case ORC_COSINE: return rf + s->amp * (1.0 - cos(w * tt));
        case ORC_STEP: return rf + s->amp;
        case ORC_RICKER: {
            /* Ricker pulse, peak frequency w / 2 pi, centred at t0 */
            double fpk = w / (2.0 * M_PI);
            double a = M_PI * fpk * (tt - s->t0);
            return rf + s->amp * (1.0 - 2.0 * a * a) * exp(-a * a);
        }
        default: return rf;
    }
}

/* ---------------------------------------------------------------- contacts */

/* Eqs. 11-12 for one pair: the contact force F (on i) and the new
 * tangential history, given the normal n (from i to j), overlap delta, the
 * contact-point relative velocity of j w.r.t. i, and the displacement time
 * increment dt (0 for a static evaluation). */
void orc_pair_force(const orc_params* p, double Ri, double Rj, const double* d_ij,
                    const double* vrel, double dt, double* ft_hist, double* F,
                    double* overlap) {
    double dist = sqrt(d_ij[0] * d_ij[0] + d_ij[1] * d_ij[1] + d_ij[2] * d_ij[2]);
    double delta = Ri + Rj - dist;
    *overlap = delta;
    if (delta <= 0) {
        F[0] = F[1] = F[2] = 0;
        ft_hist[0] = ft_hist[1] = ft_hist[2] = 0;
        return;
    }
    double n[3] = {d_ij[0] / dist, d_ij[1] / dist, d_ij[2] / dist};
    double Rs = Ri * Rj / (Ri + Rj);
    double sq = sqrt(Rs * delta);
    double kn = 2.0 * p->E_p / (3.0 * (1.0 - p->nu_p * p->nu_p));
    double kt = 2.0 * p->E_p / ((1.0 + p->nu_p) * (2.0 - p->nu_p));
    double fn_mag = kn * sq * delta;
    double vn = vrel[0] * n[0] + vrel[1] * n[1] + vrel[2] * n[2];
    double vt[3] = {vrel[0] - vn * n[0], vrel[1] - vn * n[1], vrel[2] - vn * n[2]};
    /* rotate the stored tangential force into the current tangent plane */
    double hn = ft_hist[0] * n[0] + ft_hist[1] * n[1] + ft_hist[2] * n[2];
    double ft[3];
    for (int a = 0; a < 3; ++a) ft[a] = ft_hist[a] - hn * n[a] + kt * sq * dt * vt[a];
    double ftm = sqrt(ft[0] * ft[0] + ft[1] * ft[1] + ft[2] * ft[2]);
    double cap = p->mu * fn_mag;
    if (ftm > cap) {
        double sc = cap / ftm;
        for (int a = 0; a < 3; ++a) ft[a] *= sc;
    }
    for (int a = 0; a < 3; ++a) {
        ft_hist[a] = ft[a];
        F[a] = -fn_mag * n[a] + ft[a];
    }
}

static hist_t* hist_find(hist_list* h, int j, int sx, int sy, int sz, int create) {
    for (int k = 0; k < h->n; ++k)
        if (h->e[k].j == j && h->e[k].sx == sx && h->e[k].sy == sy && h->e[k].sz == sz)
            return &h->e[k];
    if (!create) return NULL;
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 8;
        h->e = (hist_t*)realloc(h->e, sizeof(hist_t) * h->cap);
    }
    hist_t* e = &h->e[h->n++];
    e->j = j;
    e->sx = sx;
    e->sy = sy;
    e->sz = sz;
    e->ft[0] = e->ft[1] = e->ft[2] = 0;
    return e;
}

static void hist_remove(hist_list* h, hist_t* e) {
    long k = e - h->e;
    h->e[k] = h->e[h->n - 1];
    h->n--;
}

static pair_hit* pair_push(pair_list* l) {
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 8;
        l->e = (pair_hit*)realloc(l->e, sizeof(pair_hit) * l->cap);
    }
    return &l->e[l->n++];
}

/* All pairs, all periodic images (a sphere may touch several images of the
 * same neighbour when the box is narrow).  Pass 1 evaluates every pair
 * (i < j) from sphere i, which alone owns the tangential history of its
 * pairs (in parallel over i); pass 2 adds the pair forces to both spheres in
 * the order i, j, image (serially, so the sums do not depend on threads). */
static void contacts(orc_sim* s, double dt) {
    int np = s->np;
    double L[3] = {s->p.nx, s->p.ny, s->p.nz};
    int per[3] = {s->px, 1, 1};
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int i = 0; i < np; ++i) {
        s->pairs[i].n = 0;
        for (int j = i + 1; j < np; ++j) {
            double cut = s->R[i] + s->R[j];
            int lo[3], hi[3];
            for (int a = 0; a < 3; ++a) {
                if (per[a]) {
                    double dd = s->X[3 * i + a] - s->X[3 * j + a];
                    lo[a] = (int)ceil((dd - cut) / L[a]);
                    hi[a] = (int)floor((dd + cut) / L[a]);
                } else {
                    lo[a] = hi[a] = 0;
                }
            }
            for (int kx = lo[0]; kx <= hi[0]; ++kx)
                for (int ky = lo[1]; ky <= hi[1]; ++ky)
                    for (int kz = lo[2]; kz <= hi[2]; ++kz) {
                        double d[3] = {s->X[3 * j] + kx * L[0] - s->X[3 * i],
                                       s->X[3 * j + 1] + ky * L[1] - s->X[3 * i + 1],
                                       s->X[3 * j + 2] + kz * L[2] - s->X[3 * i + 2]};
                        double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                        hist_t* h = hist_find(&s->hist[i], j, kx, ky, kz, 0);
                        if (dist >= cut) {
                            if (h) hist_remove(&s->hist[i], h);
                            continue;
                        }
                        if (!h) h = hist_find(&s->hist[i], j, kx, ky, kz, 1);
                        double delta = cut - dist;
                        double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
                        double ri[3], rj[3];
                        for (int a = 0; a < 3; ++a) {
                            ri[a] = (s->R[i] - 0.5 * delta) * n[a];
                            rj[a] = -(s->R[j] - 0.5 * delta) * n[a];
                        }
                        double wi[3], wj[3], vrel[3];
                        cross(&s->Wh[3 * i], ri, wi);
                        cross(&s->Wh[3 * j], rj, wj);
                        for (int a = 0; a < 3; ++a)
                            vrel[a] = (s->Vh[3 * j + a] + wj[a]) - (s->Vh[3 * i + a] + wi[a]);
                        double F[3], ov;
                        orc_pair_force(&s->p, s->R[i], s->R[j], d, vrel, dt, h->ft, F, &ov);
                        pair_hit* e = pair_push(&s->pairs[i]);
                        double Fm[3] = {-F[0], -F[1], -F[2]};
                        e->j = j;
                        for (int a = 0; a < 3; ++a) e->F[a] = F[a];
                        cross(ri, F, e->ti);
                        cross(rj, Fm, e->tj);
                    }
        }
    }
    memset(s->Fc, 0, sizeof(double) * 3 * np);
    memset(s->Tc, 0, sizeof(double) * 3 * np);
    for (int i = 0; i < np; ++i)
        for (int k = 0; k < s->pairs[i].n; ++k) {
            const pair_hit* e = &s->pairs[i].e[k];
            int j = e->j;
            for (int a = 0; a < 3; ++a) {
                s->Fc[3 * i + a] += e->F[a];
                s->Fc[3 * j + a] -= e->F[a];
                s->Tc[3 * i + a] += e->ti[a];
                s->Tc[3 * j + a] += e->tj[a];
            }
        }
}

/* Eqs. 9-10 (spheres: I = 2/5 m R^2, no gyroscopic term), velocity Verlet
 * with K substeps of length 1/K per LBM step; hydrodynamic force/torque of
 * the LBM step held fixed; contacts re-evaluated every substep; fixed
 * spheres keep V = Omega = 0.  Quaternion: q <- normalize(q + dt/2 (0,W) q). */
static void dem_substeps(orc_sim* s) {
    int K = s->p.dem_substeps;
    double dt = 1.0 / K;
    double g[3] = {s->p.body_force[0], s->p.body_force[1], s->p.body_force[2]};
    for (int k = 0; k < K; ++k) {
        for (int i = 0; i < s->np; ++i) {
            double* Vh = &s->Vh[3 * i];
            double* Wh = &s->Wh[3 * i];
            if (s->fixed[i]) {
                Vh[0] = Vh[1] = Vh[2] = 0;
                Wh[0] = Wh[1] = Wh[2] = 0;
                continue;
            }
            for (int a = 0; a < 3; ++a) {
                Vh[a] = s->V[3 * i + a] +
                        0.5 * dt * (s->Fc[3 * i + a] + s->Fa[3 * i + a] + g[a]) / s->m[i];
                Wh[a] = s->W[3 * i + a] + 0.5 * dt * (s->Tc[3 * i + a] + s->Ta[3 * i + a]) / s->I[i];
                s->X[3 * i + a] += dt * Vh[a];
            }
            double* qq = &s->q[4 * i];
            double dq0 = -(Wh[0] * qq[1] + Wh[1] * qq[2] + Wh[2] * qq[3]);
            double wxv[3];
            cross(Wh, &qq[1], wxv);
            double dq[4] = {dq0, qq[0] * Wh[0] + wxv[0], qq[0] * Wh[1] + wxv[1],
                            qq[0] * Wh[2] + wxv[2]};
            double nq = 0;
            for (int a = 0; a < 4; ++a) {
                qq[a] += 0.5 * dt * dq[a];
                nq += qq[a] * qq[a];
            }
            nq = sqrt(nq);
            for (int a = 0; a < 4; ++a) qq[a] /= nq;
        }
        contacts(s, dt);
        for (int i = 0; i < s->np; ++i) {
            if (s->fixed[i]) {
                for (int a = 0; a < 3; ++a) s->V[3 * i + a] = s->W[3 * i + a] = 0;
                continue;
            }
            for (int a = 0; a < 3; ++a) {
                s->V[3 * i + a] = s->Vh[3 * i + a] +
                                  0.5 * dt * (s->Fc[3 * i + a] + s->Fa[3 * i + a] + g[a]) / s->m[i];
                s->W[3 * i + a] = s->Wh[3 * i + a] +
                                  0.5 * dt * (s->Tc[3 * i + a] + s->Ta[3 * i + a]) / s->I[i];
            }
        }
    }
}

/* ------------------------------------------------------------ solid map */

/* Section 2.3: a node is solid when it lies strictly inside a sphere
 * (|x - X_p|^2 < R^2, any periodic image); the inlet and outlet planes stay
 * fluid when x is not periodic.  A node inside several (touching) spheres
 * belongs to the one with the smallest |x - X_p|^2 / R_p^2, the lowest index
 * on an exact tie: each sphere then owns its own side of the contact lens,
 * and with it the fluid links around its side of the neck. */
static void paint(const orc_sim* s, int* owner) {
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    double* best = s->best;
    /* x-planes in parallel; within a plane every sphere image that reaches
     * it, in sphere order (the smallest ratio wins, ties to the lowest
     * index, so the order of the images does not matter) */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int x = 0; x < nx; ++x) {
        for (long n = nidx(s, x, 0, 0); n < nidx(s, x, 0, 0) + (long)ny * nz; ++n) owner[n] = -1;
        if (!s->px && (x == 0 || x == nx - 1)) continue;
        for (int p = 0; p < s->np; ++p) {
            double cx = s->X[3 * p], cy = s->X[3 * p + 1], cz = s->X[3 * p + 2], R = s->R[p];
            int x0 = (int)ceil(cx - R), x1 = (int)floor(cx + R);
            int y0 = (int)ceil(cy - R), y1 = (int)floor(cy + R);
            int z0 = (int)ceil(cz - R), z1 = (int)floor(cz + R);
            /* unwrapped coordinates xi in [x0, x1] that land on plane x */
            int k0 = 0, k1 = 0;
            if (s->px) {
                k0 = (int)ceil((double)(x0 - x) / nx);
                k1 = (int)floor((double)(x1 - x) / nx);
            } else if (x < x0 || x > x1) {
                continue;
            }
            for (int k = k0; k <= k1; ++k) {
                int xi = x + k * nx;
                for (int yi = y0; yi <= y1; ++yi) {
                    int y = wrapi(yi, ny);
                    for (int zi = z0; zi <= z1; ++zi) {
                        int z = wrapi(zi, nz);
                        double dx = xi - cx, dy = yi - cy, dz = zi - cz;
                        double d2 = dx * dx + dy * dy + dz * dz;
                        if (d2 < R * R) {
                            long n = nidx(s, x, y, z);
                            double ratio = d2 / (R * R);
                            if (owner[n] < 0 || ratio < best[n] || (ratio == best[n] && p < owner[n])) {
                                owner[n] = p;
                                best[n] = ratio;
                            }
                        }
                    }
                }
            }
        }
    }
}

static void lever(const orc_sim* s, double x, double y, double z, int p, double* r) {
    r[0] = minimg(x - s->X[3 * p], s->p.nx, s->px);
    r[1] = minimg(y - s->X[3 * p + 1], s->p.ny, 1);
    r[2] = minimg(z - s->X[3 * p + 2], s->p.nz, 1);
}

/* Eqs. 16-17 with the signs read as momentum bookkeeping: the particle that
 * covers a fluid node gains that node's momentum; a node that a particle
 * uncovers is rebuilt at equilibrium with the mean density rho_bar of its
 * neighbours that were fluid before the update (rho_f if none) and the
 * particle's surface velocity, and the particle loses rho_bar * V_b. */
static void update_map(orc_sim* s) {
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    paint(s, s->owner_new);
    for (int x = 0; x < nx; ++x)
        for (int y = 0; y < ny; ++y)
            for (int z = 0; z < nz; ++z) {
                long n = nidx(s, x, y, z);
                int o = s->owner[n], w = s->owner_new[n];
                if (o < 0 && w >= 0) {
                    double fm[Q], rho, j[3], r[3], t[3];
                    for (int m = 0; m < Q; ++m) fm[m] = s->f[m * s->N + n];
                    moments(fm, &rho, j);
                    lever(s, x, y, z, w, r);
                    cross(r, j, t);
                    for (int a = 0; a < 3; ++a) {
                        s->Fh[3 * w + a] += j[a];
                        s->Th[3 * w + a] += t[a];
                    }
                } else if (o >= 0 && w < 0) {
                    double sum = 0;
                    int cnt = 0;
                    for (int m = 0; m < Q; ++m) {
                        if (CX[m] == 0 && CY[m] == 0 && CZ[m] == 0) continue;
                        int xx = x + CX[m];
                        if (s->px) xx = wrapi(xx, nx);
                        else if (xx < 0 || xx >= nx) continue;
                        long k = nidx(s, xx, wrapi(y + CY[m], ny), wrapi(z + CZ[m], nz));
                        if (s->owner[k] >= 0) continue;
                        double rr = 0;
                        for (int mm = 0; mm < Q; ++mm) rr += s->f[mm * s->N + k];
                        sum += rr;
                        cnt++;
                    }
                    double rb = cnt ? sum / cnt : s->p.rho_f;
                    double r[3], wr[3], Vb[3], feq[Q], t[3], mom[3];
                    lever(s, x, y, z, o, r);
                    cross(&s->W[3 * o], r, wr);
                    for (int a = 0; a < 3; ++a) Vb[a] = s->V[3 * o + a] + wr[a];
                    orc_equilibrium(rb, Vb[0], Vb[1], Vb[2], feq);
                    for (int m = 0; m < Q; ++m) s->f[m * s->N + n] = feq[m];
                    for (int a = 0; a < 3; ++a) mom[a] = rb * Vb[a];
                    cross(r, mom, t);
                    for (int a = 0; a < 3; ++a) {
                        s->Fh[3 * o + a] -= mom[a];
                        s->Th[3 * o + a] -= t[a];
                    }
                }
            }
    int* tmp = s->owner;
    s->owner = s->owner_new;
    s->owner_new = tmp;
}

/* ------------------------------------------------------------ LBM step */

static void lbm_step(orc_sim* s) {
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    long N = s->N;
    double tau = s->p.tau, rf = s->p.rho_f;
    memset(s->Fh, 0, sizeof(double) * 3 * s->np);
    memset(s->Th, 0, sizeof(double) * 3 * s->np);
    update_map(s);

    /* probe: mean density over fluid nodes of plane probe_x, entering the
     * collision of this step (Section 3.2 averages over fluid nodes only) */
    if (s->p.probe_x >= 0 && s->p.probe_x < nx) {
        double sum = 0;
        long cnt = 0;
        for (int y = 0; y < ny; ++y)
            for (int z = 0; z < nz; ++z) {
                long n = nidx(s, s->p.probe_x, y, z);
                if (s->owner[n] >= 0) continue;
                for (int m = 0; m < Q; ++m) sum += s->f[m * N + n];
                cnt++;
            }
        if (s->trace_len == s->trace_cap) {
            s->trace_cap = s->trace_cap ? 2 * s->trace_cap : 1024;
            s->trace = (double*)realloc(s->trace, sizeof(double) * s->trace_cap);
        }
        s->trace[s->trace_len++] = cnt ? sum / cnt : NAN;
    }

    /* collision, Eq. 4 (node by node; independent) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (long n = 0; n < N; ++n) {
        if (s->owner[n] >= 0) continue;
        double fm[Q];
        for (int m = 0; m < Q; ++m) fm[m] = s->f[m * N + n];
        orc_collide_node(fm, tau);
        for (int m = 0; m < Q; ++m) s->f[m * N + n] = fm[m];
    }

    /* streaming, Eq. 5, with half-way bounce-back, Eqs. 14-15.  Every
     * target slot has exactly one writer (the upstream node, or the node
     * itself when the upstream neighbour is solid or outside), so the
     * x-planes stream in parallel; the link force and torque of each plane
     * are summed in that plane's list and the lists added in x order. */
    const int np = s->np;
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        double* acc = (double*)calloc(6 * (size_t)(np > 0 ? np : 1), sizeof(double));
        int* touched = (int*)malloc(sizeof(int) * (size_t)(np > 0 ? np : 1));
        unsigned char* mark = (unsigned char*)calloc((size_t)(np > 0 ? np : 1), 1);
        /* the new lattice starts from zero (solid nodes keep zeros); the
         * implicit barrier of the loop separates this from the streaming */
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int x = 0; x < nx; ++x)
            for (int m = 0; m < Q; ++m)
                memset(&s->fn[m * N + nidx(s, x, 0, 0)], 0, sizeof(double) * (size_t)ny * nz);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int x = 0; x < nx; ++x) {
            int nt = 0;
            for (int y = 0; y < ny; ++y)
                for (int z = 0; z < nz; ++z) {
                    long n = nidx(s, x, y, z);
                    if (s->owner[n] >= 0) continue;
                    for (int m = 0; m < Q; ++m) {
                        double ft = s->f[m * N + n];
                        int xx = x + CX[m];
                        if (s->px) {
                            xx = wrapi(xx, nx);
                        } else if (xx < 0 || xx >= nx) {
                            s->fn[OPP[m] * N + n] = ft;
                            continue;
                        }
                        long k = nidx(s, xx, wrapi(y + CY[m], ny), wrapi(z + CZ[m], nz));
                        int p = s->owner[k];
                        if (p < 0) {
                            s->fn[m * N + k] = ft;
                            continue;
                        }
                        double xb = x + 0.5 * CX[m], yb = y + 0.5 * CY[m], zb = z + 0.5 * CZ[m];
                        double r[3], wr[3], Vb[3];
                        lever(s, xb, yb, zb, p, r);
                        cross(&s->W[3 * p], r, wr);
                        for (int a = 0; a < 3; ++a) Vb[a] = s->V[3 * p + a] + wr[a];
                        double cv = CX[m] * Vb[0] + CY[m] * Vb[1] + CZ[m] * Vb[2];
                        /* Eq. 14 with rho_w = rho_f and 2 w / c_s^2 = 6 w */
                        double back = ft - 6.0 * WT[m] * rf * cv;
                        s->fn[OPP[m] * N + n] = back;
                        /* Eq. 15 taken about the rest state: the mean pressure
                         * rho_f c_s^2 acts on the whole grain (the granular
                         * stress of Eq. 13 is an effective stress), so the
                         * exchanged momentum is counted from 2 w rho_f; the
                         * literal form (link_literal) omits that reference */
                        double q = ft + back - (s->link_literal ? 0.0 : 2.0 * WT[m] * rf);
                        double Fl[3] = {CX[m] * q, CY[m] * q, CZ[m] * q};
                        double t[3];
                        cross(r, Fl, t);
                        if (!mark[p]) {
                            mark[p] = 1;
                            touched[nt++] = p;
                        }
                        for (int a = 0; a < 3; ++a) {
                            acc[6 * p + a] += Fl[a];
                            acc[6 * p + 3 + a] += t[a];
                        }
                    }
                }
            plane_list* pl = &s->plane_acc[x];
            pl->n = 0;
            if (nt > pl->cap) {
                pl->cap = nt;
                pl->e = (plane_sum*)realloc(pl->e, sizeof(plane_sum) * nt);
            }
            for (int k = 0; k < nt; ++k) {
                int p = touched[k];
                plane_sum* e = &pl->e[pl->n++];
                e->p = p;
                for (int a = 0; a < 3; ++a) {
                    e->F[a] = acc[6 * p + a];
                    e->T[a] = acc[6 * p + 3 + a];
                }
                for (int a = 0; a < 6; ++a) acc[6 * p + a] = 0.0;
                mark[p] = 0;
            }
        }
        free(acc);
        free(touched);
        free(mark);
    }
    for (int x = 0; x < nx; ++x)
        for (int k = 0; k < s->plane_acc[x].n; ++k) {
            const plane_sum* e = &s->plane_acc[x].e[k];
            for (int a = 0; a < 3; ++a) {
                s->Fh[3 * e->p + a] += e->F[a];
                s->Th[3 * e->p + a] += e->T[a];
            }
        }

    /* inlet and outlet (Section 2.4; Eq. 25 evaluated at the new time) */
    if (!s->px) {
        long long tn = s->t + 1;
        if (s->p.inlet == ORC_INLET_PRESSURE) {
            double rin = orc_source_density(s, tn);
            for (int y = 0; y < ny; ++y)
                for (int z = 0; z < nz; ++z) {
                    long n = nidx(s, 0, y, z);
                    double fm[Q];
                    for (int m = 0; m < Q; ++m) fm[m] = s->fn[m * N + n];
                    orc_pressure_face(fm, rin, 0);
                    for (int m = 0; m < Q; ++m) s->fn[m * N + n] = fm[m];
                }
        }
        if (s->p.outlet == ORC_OUTLET_ZERO_GRADIENT && nx >= 2) {
            for (int y = 0; y < ny; ++y)
                for (int z = 0; z < nz; ++z) {
                    long n = nidx(s, nx - 1, y, z), u = nidx(s, nx - 2, y, z);
                    if (s->owner[u] >= 0) continue;
                    for (int m = 0; m < Q; ++m)
                        if (CX[m] == -1) s->fn[m * N + n] = s->fn[m * N + u];
                }
        } else if (s->p.outlet == ORC_OUTLET_PRESSURE) {
            for (int y = 0; y < ny; ++y)
                for (int z = 0; z < nz; ++z) {
                    long n = nidx(s, nx - 1, y, z);
                    double fm[Q];
                    for (int m = 0; m < Q; ++m) fm[m] = s->fn[m * N + n];
                    orc_pressure_face(fm, rf, 1);
                    for (int m = 0; m < Q; ++m) s->fn[m * N + n] = fm[m];
                }
        }
    }
    double* tmp = s->f;
    s->f = s->fn;
    s->fn = tmp;
}

/* ------------------------------------------------------------ surrogate */

/* Smooth solid fraction of a node (a C1 stand-in for the binary solid map,
 * the surrogate's only dependence on the sphere centres): sphere p covers
 * eps_p = S(R_p - |x - X_p| + 1/2) of the node, S the cubic smoothstep
 * (0 below 0, 3 s^2 - 2 s^3 on [0, 1], 1 above), the distance taken to the
 * nearest periodic image; overlapping spheres combine as
 * eps = 1 - prod_p (1 - eps_p).  The x planes 0 and nx-1 stay fluid when x
 * is not periodic (as in the solid map). */
static double smoothstep(double v) {
    if (v <= 0.0) return 0.0;
    if (v >= 1.0) return 1.0;
    return v * v * (3.0 - 2.0 * v);
}

static double psm_fraction_at(const orc_sim* s, int x, int y, int z) {
    if (!s->px && (x == 0 || x == s->p.nx - 1)) return 0.0;
    double keep = 1.0;
    for (int p = 0; p < s->np; ++p) {
        double r[3];
        lever(s, x, y, z, p, r);
        double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        keep *= 1.0 - smoothstep(s->R[p] - d + 0.5);
    }
    return 1.0 - keep;
}

void orc_psm_fraction(const orc_sim* s, double* eps) {
    for (int x = 0; x < s->p.nx; ++x)
        for (int y = 0; y < s->p.ny; ++y)
            for (int z = 0; z < s->p.nz; ++z)
                eps[nidx(s, x, y, z)] = s->eps ? s->eps[nidx(s, x, y, z)] : psm_fraction_at(s, x, y, z);
}

/* One step of the surrogate, in the order of lbm_step: at every node the
 * Noble-Torczynski collision with solid fraction eps and a resting solid,
 *   f*_i = f_i - (1 - B)/tau (f_i - f^eq_i) + B Om_i,
 *   B = eps (tau - 1/2) / ((1 - eps) + (tau - 1/2)),
 *   Om_i = f_opp(i) - f_i + w_i rho - f^eq_opp(i)(rho, u)
 * (the bounce-back of the non-equilibrium part), then plain streaming
 * (every node carries populations; populations leaving the x range come
 * back reversed, as at a resting wall), then the inlet and outlet of
 * lbm_step.  The probe averages the density over every node of its plane. */
static void psm_step(orc_sim* s) {
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    long N = s->N;
    double tau = s->p.tau, sh = tau - 0.5;
    if (!s->eps && !s->eps_auto) {
        s->eps_auto = (double*)malloc(sizeof(double) * N);
        orc_psm_fraction(s, s->eps_auto);
    }
    const double* epsv = s->eps ? s->eps : s->eps_auto;
    if (s->p.probe_x >= 0 && s->p.probe_x < nx) {
        double sum = 0;
        for (int y = 0; y < ny; ++y)
            for (int z = 0; z < nz; ++z) {
                long n = nidx(s, s->p.probe_x, y, z);
                for (int m = 0; m < Q; ++m) sum += s->f[m * N + n];
            }
        if (s->trace_len == s->trace_cap) {
            s->trace_cap = s->trace_cap ? 2 * s->trace_cap : 1024;
            s->trace = (double*)realloc(s->trace, sizeof(double) * s->trace_cap);
        }
        s->trace[s->trace_len++] = sum / ((double)ny * nz);
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int x = 0; x < nx; ++x)
        for (int y = 0; y < ny; ++y)
            for (int z = 0; z < nz; ++z) {
                long n = nidx(s, x, y, z);
                double eps = epsv[n];
                double B = eps * sh / ((1.0 - eps) + sh);
                double fm[Q], rho, j[3], feq[Q], fs[Q];
                for (int m = 0; m < Q; ++m) fm[m] = s->f[m * N + n];
                moments(fm, &rho, j);
                orc_equilibrium(rho, j[0] / rho, j[1] / rho, j[2] / rho, feq);
                for (int m = 0; m < Q; ++m) {
                    double om = fm[OPP[m]] - fm[m] + WT[m] * rho - feq[OPP[m]];
                    fs[m] = fm[m] - (1.0 - B) / tau * (fm[m] - feq[m]) + B * om;
                }
                for (int m = 0; m < Q; ++m) {
                    int xx = x + CX[m];
                    if (s->px) {
                        xx = wrapi(xx, nx);
                    } else if (xx < 0 || xx >= nx) {
                        s->fn[OPP[m] * N + n] = fs[m];
                        continue;
                    }
                    s->fn[m * N + nidx(s, xx, wrapi(y + CY[m], ny), wrapi(z + CZ[m], nz))] = fs[m];
                }
            }
    if (!s->px) {
        long long tn = s->t + 1;
        if (s->p.inlet == ORC_INLET_PRESSURE) {
            double rin = orc_source_density(s, tn);
            for (int y = 0; y < ny; ++y)
                for (int z = 0; z < nz; ++z) {
                    long n = nidx(s, 0, y, z);
                    double fm[Q];
                    for (int m = 0; m < Q; ++m) fm[m] = s->fn[m * N + n];
                    orc_pressure_face(fm, rin, 0);
                    for (int m = 0; m < Q; ++m) s->fn[m * N + n] = fm[m];
                }
        }
        if (s->p.outlet == ORC_OUTLET_ZERO_GRADIENT && nx >= 2) {
            for (int y = 0; y < ny; ++y)
                for (int z = 0; z < nz; ++z) {
                    long n = nidx(s, nx - 1, y, z), u = nidx(s, nx - 2, y, z);
                    for (int m = 0; m < Q; ++m)
                        if (CX[m] == -1) s->fn[m * N + n] = s->fn[m * N + u];
                }
        } else if (s->p.outlet == ORC_OUTLET_PRESSURE) {
            for (int y = 0; y < ny; ++y)
                for (int z = 0; z < nz; ++z) {
                    long n = nidx(s, nx - 1, y, z);
                    double fm[Q];
                    for (int m = 0; m < Q; ++m) fm[m] = s->fn[m * N + n];
                    orc_pressure_face(fm, s->p.rho_f, 1);
                    for (int m = 0; m < Q; ++m) s->fn[m * N + n] = fm[m];
                }
        }
    }
    double* tmp = s->f;
    s->f = s->fn;
    s->fn = tmp;
}

void orc_set_coupling(orc_sim* s, int psm) { s->psm = psm ? 1 : 0; }

void orc_psm_set_fraction(orc_sim* s, const double* eps) {
    free(s->eps);
    s->eps = NULL;
    if (!eps) return;
    s->eps = (double*)malloc(sizeof(double) * s->N);
    memcpy(s->eps, eps, sizeof(double) * s->N);
}

/* ------------------------------------------------------------ public API */

orc_sim* orc_create(const orc_params* p) {
    init_tables();
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->tau <= 0.5 || p->dem_substeps < 1) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->px = (p->inlet == ORC_X_PERIODIC);
    s->N = (long)p->nx * p->ny * p->nz;
    s->f = (double*)malloc(sizeof(double) * Q * s->N);
    s->fn = (double*)malloc(sizeof(double) * Q * s->N);
    s->owner = (int*)malloc(sizeof(int) * s->N);
    s->owner_new = (int*)malloc(sizeof(int) * s->N);
    s->best = (double*)malloc(sizeof(double) * s->N);
    s->plane_acc = (plane_list*)calloc((size_t)p->nx, sizeof(plane_list));
    if (!s->f || !s->fn || !s->owner || !s->owner_new || !s->best || !s->plane_acc) {
        orc_destroy(s);
        return NULL;
    }
    double feq[Q];
    orc_equilibrium(p->rho_f, 0, 0, 0, feq);
    for (int m = 0; m < Q; ++m)
        for (long n = 0; n < s->N; ++n) s->f[m * s->N + n] = feq[m];
    for (long n = 0; n < s->N; ++n) s->owner[n] = -1;
    s->waveform = ORC_SINE;
    s->amp = 0;
    s->t_n = -1;
    return s;
}

int orc_set_packing(orc_sim* s, int n, const double* X, const double* R, const double* V,
                    const double* W, const unsigned char* fixed) {
    free(s->X);
    free(s->V);
    free(s->W);
    free(s->q);
    free(s->R);
    free(s->m);
    free(s->I);
    free(s->fixed);
    free(s->Fh);
    free(s->Th);
    free(s->Fc);
    free(s->Tc);
    free(s->Vh);
    free(s->Wh);
    free(s->Fh_prev);
    free(s->Th_prev);
    free(s->Fa);
    free(s->Ta);
    if (s->hist) {
        for (int i = 0; i < s->np; ++i) free(s->hist[i].e);
        free(s->hist);
    }
    if (s->pairs) {
        for (int i = 0; i < s->np; ++i) free(s->pairs[i].e);
        free(s->pairs);
    }
    free(s->eps_auto);
    s->eps_auto = NULL;
    s->np = n;
    int nn = n > 0 ? n : 1;
    s->X = (double*)calloc(3 * nn, sizeof(double));
    s->V = (double*)calloc(3 * nn, sizeof(double));
    s->W = (double*)calloc(3 * nn, sizeof(double));
    s->q = (double*)calloc(4 * nn, sizeof(double));
    s->R = (double*)calloc(nn, sizeof(double));
    s->m = (double*)calloc(nn, sizeof(double));
    s->I = (double*)calloc(nn, sizeof(double));
    s->fixed = (unsigned char*)calloc(nn, 1);
    s->Fh = (double*)calloc(3 * nn, sizeof(double));
    s->Th = (double*)calloc(3 * nn, sizeof(double));
    s->Fc = (double*)calloc(3 * nn, sizeof(double));
    s->Tc = (double*)calloc(3 * nn, sizeof(double));
    s->Vh = (double*)calloc(3 * nn, sizeof(double));
    s->Wh = (double*)calloc(3 * nn, sizeof(double));
    s->Fh_prev = (double*)calloc(3 * nn, sizeof(double));
    s->Th_prev = (double*)calloc(3 * nn, sizeof(double));
    s->Fa = (double*)calloc(3 * nn, sizeof(double));
    s->Ta = (double*)calloc(3 * nn, sizeof(double));
    s->hist = (hist_list*)calloc(nn, sizeof(hist_list));
    s->pairs = (pair_list*)calloc(nn, sizeof(pair_list));
    for (int i = 0; i < n; ++i) {
        if (!(R[i] > 0)) return -1;
        for (int a = 0; a < 3; ++a) {
            s->X[3 * i + a] = X[3 * i + a];
            s->V[3 * i + a] = V ? V[3 * i + a] : 0.0;
            s->W[3 * i + a] = W ? W[3 * i + a] : 0.0;
        }
        s->fixed[i] = fixed ? fixed[i] : 0;
        if (s->fixed[i])
            for (int a = 0; a < 3; ++a) s->V[3 * i + a] = s->W[3 * i + a] = 0;
        s->q[4 * i] = 1.0;
        s->R[i] = R[i];
        s->m[i] = s->p.rho_p * 4.0 / 3.0 * M_PI * R[i] * R[i] * R[i];
        s->I[i] = 0.4 * s->m[i] * R[i] * R[i];
    }
    /* fluid at rest at rho_f, solid map painted, initial contacts with zero
     * tangential history */
    double feq[Q];
    orc_equilibrium(s->p.rho_f, 0, 0, 0, feq);
    for (int m = 0; m < Q; ++m)
        for (long k = 0; k < s->N; ++k) s->f[m * s->N + k] = feq[m];
    paint(s, s->owner);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            s->Vh[3 * i + a] = s->V[3 * i + a];
            s->Wh[3 * i + a] = s->W[3 * i + a];
        }
    contacts(s, 0.0);
    s->t = 0;
    s->trace_len = 0;
    s->have_packing = 1;
    return 0;
}

int orc_set_source(orc_sim* s, int waveform, double amplitude, double omega, long long t_n,
                   double t0) {
    if (waveform < 0 || waveform > ORC_RICKER) return -1;
    s->waveform = waveform;
    s->amp = amplitude;
    s->omega = omega;
    s->t_n = t_n;
    s->t0 = t0;
    return 0;
}

int orc_step(orc_sim* s, long long nsteps) {
    if (!s->have_packing) return -1;
    for (long long k = 0; k < nsteps; ++k) {
        if (s->p.lbm_on && s->psm) {
            memset(s->Fh, 0, sizeof(double) * 3 * s->np);
            memset(s->Th, 0, sizeof(double) * 3 * s->np);
            psm_step(s);
        } else if (s->p.lbm_on) {
            lbm_step(s);
        } else {
            memset(s->Fh, 0, sizeof(double) * 3 * s->np);
            memset(s->Th, 0, sizeof(double) * 3 * s->np);
        }
        for (int i = 0; i < 3 * s->np; ++i) {
            s->Fa[i] = 0.5 * (s->Fh[i] + s->Fh_prev[i]);
            s->Ta[i] = 0.5 * (s->Th[i] + s->Th_prev[i]);
            s->Fh_prev[i] = s->Fh[i];
            s->Th_prev[i] = s->Th[i];
        }
        dem_substeps(s);
        s->t++;
    }
    return 0;
}

long long orc_time(const orc_sim* s) { return s->t; }

void orc_fields(const orc_sim* s, double* rho, double* u, unsigned char* solid) {
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        int sol = s->owner[n] >= 0 && !s->psm;
        if (solid) solid[n] = (unsigned char)sol;
        double fm[Q], r = 0, j[3] = {0, 0, 0};
        if (!sol) {
            for (int m = 0; m < Q; ++m) fm[m] = s->f[m * N + n];
            moments(fm, &r, j);
        }
        if (rho) rho[n] = sol ? 0.0 : r;
        if (u)
            for (int a = 0; a < 3; ++a) u[a * N + n] = sol ? 0.0 : j[a] / r;
    }
}

void orc_populations(const orc_sim* s, double* f) { memcpy(f, s->f, sizeof(double) * Q * s->N); }

void orc_set_populations(orc_sim* s, const double* f) {
    memcpy(s->f, f, sizeof(double) * Q * s->N);
}

void orc_owner(const orc_sim* s, int* owner) { memcpy(owner, s->owner, sizeof(int) * s->N); }

void orc_particles(const orc_sim* s, double* X, double* V, double* W, double* q, double* Fh,
                   double* Th) {
    int n = s->np;
    if (X) memcpy(X, s->X, sizeof(double) * 3 * n);
    if (V) memcpy(V, s->V, sizeof(double) * 3 * n);
    if (W) memcpy(W, s->W, sizeof(double) * 3 * n);
    if (q) memcpy(q, s->q, sizeof(double) * 4 * n);
    if (Fh) memcpy(Fh, s->Fh, sizeof(double) * 3 * n);
    if (Th) memcpy(Th, s->Th, sizeof(double) * 3 * n);
}

void orc_contact_forces(const orc_sim* s, double* Fc, double* Tc) {
    if (Fc) memcpy(Fc, s->Fc, sizeof(double) * 3 * s->np);
    if (Tc) memcpy(Tc, s->Tc, sizeof(double) * 3 * s->np);
}

long long orc_probe(const orc_sim* s, double* trace, long long max_len) {
    long long n = s->trace_len < max_len ? s->trace_len : max_len;
    if (trace && n > 0) memcpy(trace, s->trace, sizeof(double) * n);
    return s->trace_len;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->f);
    free(s->fn);
    free(s->owner);
    free(s->owner_new);
    free(s->best);
    free(s->X);
    free(s->V);
    free(s->W);
    free(s->q);
    free(s->R);
    free(s->m);
    free(s->I);
    free(s->fixed);
    free(s->Fh);
    free(s->Th);
    free(s->Fc);
    free(s->Tc);
    free(s->Vh);
    free(s->Wh);
    free(s->Fh_prev);
    free(s->Th_prev);
    free(s->Fa);
    free(s->Ta);
    if (s->hist) {
        for (int i = 0; i < s->np; ++i) free(s->hist[i].e);
        free(s->hist);
    }
    if (s->pairs) {
        for (int i = 0; i < s->np; ++i) free(s->pairs[i].e);
        free(s->pairs);
    }
    if (s->plane_acc) {
        for (int x = 0; x < s->p.nx; ++x) free(s->plane_acc[x].e);
        free(s->plane_acc);
    }
    free(s->trace);
    free(s->eps);
    free(s->eps_auto);
    free(s);
}

void orc_set_link_form(orc_sim* s, int literal) { s->link_literal = literal ? 1 : 0; }

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
