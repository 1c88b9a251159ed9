/*
 * art_oracle.h -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * Declarations of the plain FP64 CPU oracle for adaptive ray tracing of Kerr black-hole images
 * (Gelles et al. 2021, "The Role of Adaptive Ray Tracing in Analyzing Black Hole Structure").
 * Only the test suite, the package smoke check and the CPU-baseline leg of the benchmark may
 * load this library.  It shares no code, header or table with the CUDA library.
 */
#ifndef ART_ORACLE_H
#define ART_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Emission models. */
enum { ORC_EMIT_ANALYTIC = 0,      /* j = r^-2 exp(-z^2/(2 (w r)^2)), Keplerian flow, no absorption */
       ORC_EMIT_SYNCH_DISK = 1,/* thermal synchrotron thin disk, polarized (Stokes IQUV)       */
       ORC_EMIT_GRID = 2,      /* thermal synchrotron from a fluid grid (rho, u, u^i, B^i)      */
       ORC_EMIT_BLOB = 8 };    /* flat-space test: static Gaussian blob, sigma = blob_sigma    */
enum { ORC_FLOW_KEPLER = 0, ORC_FLOW_STATIC = 1 };
enum { ORC_NORM_IBAR_INT = 0, ORC_NORM_PEAK = 1 };
enum { ORC_INTERP_LINEAR = 0, ORC_INTERP_NEAREST = 1 };
enum { ORC_EDGE_ONESIDED = 0, ORC_EDGE_TRACE = 1 };
enum { ORC_RAY_ESCAPED = 0, ORC_RAY_CAPTURED = 1, ORC_RAY_CAP = 2, ORC_RAY_NAN = 3 };
enum { ORC_MASK_UNSET = 0, ORC_MASK_TRACED = 1, ORC_MASK_INTERP = 2 };

typedef struct orc_job {
    double a;            /* dimensionless spin */
    double mass;         /* M (1 in all production configurations, 0 for flat-space checks) */
    double r_obs;        /* camera radius (M) */
    double incl_deg;     /* camera inclination (deg) */
    double fov;          /* horizontal field of view (M); pixel spacing = fov/(nx-1) on both axes */
    int n0x, n0y;        /* base grid */
    int levels;          /* N refinement levels */
    double R_rel, R_abs; /* tolerances */
    int abs_norm;        /* ORC_NORM_* */
    int interp;          /* ORC_INTERP_* */
    int edge_mode;       /* ORC_EDGE_* */
    int emission;        /* ORC_EMIT_* */
    int flow;            /* ORC_FLOW_* */
    int stokes;          /* 1 or 4 */
    int subrings;        /* 0 = no decomposition, else number of subring planes */
    int max_steps;
    double step_frac;    /* RK4 step h = step_frac * r */
    double h_min;        /* floor on h */
    double horizon_eps;  /* stop inward rays at r < (1+horizon_eps) r_+ */
    double escape_frac;  /* stop outgoing rays at r > escape_frac * r_obs */
    double disk_w;       /* vertical Gaussian width (fraction of r) of the emissivity */
    double blob_sigma;   /* flat-space blob width */
    /* thermal-synchrotron disk (ORC_EMIT_SYNCH_DISK) */
    double ne0, thetae0, b0, nu_hz, ne_slope, te_slope, r_in;
    double length_cm;    /* GM/c^2 in cm (converts affine lengths to cm) */
    double bz_ratio;     /* vertical / toroidal field ratio of the disk (1 = 1:1) */
    /* fluid grid (ORC_EMIT_GRID): cells (k, j, i) over phi, theta, ln r stored as
     * grid[((k * gn2 + j) * gn1 + i) * 8 + q], q = rho, u, u^r, u^theta, u^phi, B^r, B^theta,
     * B^phi (Kerr-Schild spherical components); cell centres at
     * ln r = glogr_min + (i + 1/2) dx1, theta = (j + 1/2) pi/gn2, phi = (k + 1/2) 2 pi/gn3 */
    const float* grid;
    int gn1, gn2, gn3, gpad;
    double glogr_min, glogr_max;
    double gamma_ad;     /* adiabatic index of the fluid */
    double m_unit;       /* mass unit (g): rho_cgs = rho m_unit / length_cm^3 */
    double r_high, r_low;/* ion-to-electron temperature ratio at high / low plasma beta */
    double sigma_cut;    /* no emission where b^2/rho > sigma_cut */
    int criterion;       /* ORC_CRIT_I: decide on I; ORC_CRIT_STOKES_ANY: trace when the
                          * criterion holds for any of I, Q, U, V (stokes = 4) */
    int criterion_plane; /* the plane the criterion reads (subring n: plane n * stokes) */
} orc_job;
enum { ORC_CRIT_I = 0, ORC_CRIT_STOKES_ANY = 1 };

typedef struct orc_rayinfo {
    int32_t status, steps, nturn, pad;
    double min_r, lam, eta;
} orc_rayinfo;

typedef struct orc_stats {
    int64_t rays_traced, steps;
    int64_t rays_per_level[16];
    double ibar;
} orc_stats;

int    orc_image_size(const orc_job* job, int* nx, int* ny);
int    orc_planes(const orc_job* job);
void   orc_set_threads(int n);
int    orc_get_threads(void);
int    orc_trace_screen(const orc_job* job, int n, const double* alpha, const double* beta,
                        double* out, orc_rayinfo* info);
int    orc_trace_pixels(const orc_job* job, int n, const int64_t* pix, double* out,
                        orc_rayinfo* info);
int    orc_trace_record(const orc_job* job, double alpha, double beta, int maxrec,
                        double* rec, int* nrec);
double orc_bessel_k(int n, double x);
int    orc_synch_coeffs(double ne, double thetae, double B, double nu, double theta_b,
                        double* out7);
void   orc_segment(const double* K7, const double* J4, double h, double* E16, double* X4);
void   orc_transport_rhs(const orc_job* job, const double* y12, double* df4);
void   orc_coefficients(const orc_job* job, const double* y12, int pol, double* J4, double* K7);
int    orc_grid_fluid(const orc_job* job, const double* x, double* prim8, double* u4, double* b4,
                      double* plasma4);
int    orc_emission(const orc_job* job, const double* x, const double* k, double* jnu,
                    double* nu_fl);
double orc_ibar_int(const double* img, int nx, int ny, int stride);
int    orc_refine_level(const orc_job* job, double* img, uint8_t* mask, int nx, int ny,
                        int level, double norm, double* est_abs, double* est_rel);
int    orc_render(const orc_job* job, const double* truth, double* img, uint8_t* mask,
                  orc_stats* stats);
void   orc_metrics(const double* truth, const double* img, const uint8_t* mask, int nx, int ny,
                   double* out);

#ifdef __cplusplus
}
#endif
#endif
