/*
 * lbmdem_oracle.h -- interface of the FP64 CPU reference (test
 * infrastructure only; see lbmdem_oracle.c).  Independent of the product
 * library's header: nothing here is shared with the CUDA path.
 */
#ifndef LBMDEM_ORACLE_H
#define LBMDEM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SINE = 0, ORC_COSINE = 1, ORC_STEP = 2, ORC_RICKER = 3 };
enum { ORC_INLET_PRESSURE = 0, ORC_X_WALL = 1, ORC_X_PERIODIC = 2 };
enum { ORC_OUTLET_ZERO_GRADIENT = 0, ORC_OUTLET_PRESSURE = 1, ORC_OUTLET_WALL = 2 };

typedef struct {
    int nx, ny, nz;       /* lattice; x = propagation axis */
    double tau, rho_f;    /* Eq. 4 relaxation time, mean density */
    int inlet;            /* ORC_INLET_PRESSURE | ORC_X_WALL | ORC_X_PERIODIC */
    int outlet;           /* ORC_OUTLET_* (ignored when x is periodic) */
    int dem_substeps;     /* K >= 1 */
    double E_p, nu_p, mu, rho_p; /* Eqs. 11-12, Table 1 */
    double body_force[3]; /* F_g of Eq. 9 on every free sphere */
    int probe_x;          /* plane of the density probe, -1 = off */
    int lbm_on;           /* 0: DEM only */
} orc_params;

typedef struct orc_sim orc_sim;

orc_sim* orc_create(const orc_params* p);
int orc_set_packing(orc_sim* s, int n, const double* X, const double* R, const double* V,
                    const double* W, const unsigned char* fixed);
int orc_set_source(orc_sim* s, int waveform, double amplitude, double omega, long long t_n,
                   double t0);
int orc_step(orc_sim* s, long long nsteps);
long long orc_time(const orc_sim* s);
void orc_fields(const orc_sim* s, double* rho, double* u, unsigned char* solid);
void orc_populations(const orc_sim* s, double* f);
void orc_set_populations(orc_sim* s, const double* f);
void orc_owner(const orc_sim* s, int* owner);
void orc_particles(const orc_sim* s, double* X, double* V, double* W, double* q, double* Fh,
                   double* Th);
void orc_contact_forces(const orc_sim* s, double* Fc, double* Tc);
long long orc_probe(const orc_sim* s, double* trace, long long max_len);
void orc_destroy(orc_sim* s);

/* 1: count the link momentum as printed in Eq. 15, c_d (f~_d + f_d*);
 * 0 (default): about the rest state, c_d (f~_d + f_d* - 2 w_d rho_f). */
void orc_set_link_form(orc_sim* s, int literal);
/* 1: the smooth partially-saturated surrogate coupling for gradients in the
 * sphere positions (fixed spheres; outside the paper's chosen method);
 * 0 (default): the momentum-exchange coupling. */
void orc_set_coupling(orc_sim* s, int psm);
/* The surrogate's solid fraction of every node [x][y][z]; a non-NULL eps
 * given to orc_psm_set_fraction replaces it (NULL restores it). */
void orc_psm_fraction(const orc_sim* s, double* eps);
void orc_psm_set_fraction(orc_sim* s, const double* eps);
/* OpenMP threads of every later call (results do not depend on it). */
void orc_set_threads(int n);
int orc_get_threads(void);

/* single-node pieces, exposed for the pins */
void orc_lattice(int* cx, int* cy, int* cz, double* w, int* opp);
void orc_equilibrium(double rho, double ux, double uy, double uz, double* feq);
void orc_collide_node(double* fm, double tau);
void orc_pressure_face(double* fm, double rho_b, int side);
double orc_source_density(const orc_sim* s, long long t);
void orc_pair_force(const orc_params* p, double Ri, double Rj, const double* d_ij,
                    const double* vrel, double dt, double* ft_hist, double* F, double* overlap);

#ifdef __cplusplus
}
#endif
#endif
