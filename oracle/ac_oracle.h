/*
 * ac_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure
 * only; see ac_oracle.c).  This header is private to oracle/: the CUDA library
 * has its own, unrelated declarations.
 */
#ifndef AC_ORACLE_H
#define AC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_ERR_NONFINITE = -3 };
enum { ORC_BC_WALL_SLIP = 0, ORC_BC_WALL_NOSLIP = 1, ORC_BC_TRANSMISSIVE = 2, ORC_BC_PERIODIC = 3 };
enum { ORC_RIEMANN_OSHER = 0, ORC_RIEMANN_BASSI = 1, ORC_RIEMANN_ROE = 2 };
enum {
    ORC_GRADP_NEW = 0,
    ORC_GRADP_MINMOD = 1,
    ORC_GRADP_SUPERBEE = 2,
    ORC_GRADP_SPLIT_MINMOD = 3,
    ORC_GRADP_SPLIT_SUPERBEE = 4
};

typedef struct {
    int nx, ny;            /* interior cells */
    double dx, dy;         /* cell sizes (m) */
    double gx, gy;         /* gravity (m/s^2) */
    double beta;           /* artificial compressibility (Pa) */
    int bc[4];             /* x-lo, x-hi, y-lo, y-hi */
    int s_max;             /* Runge-Kutta stages */
    int riemann;           /* ORC_RIEMANN_* */
    int gradp;             /* ORC_GRADP_* */
    int limiter_k;         /* k of the limiter for rho, u, v (1 minmod, 2 superbee) */
    int local_dtau;        /* 1 local, 0 global pseudo-time step */
    int realtime;          /* 1: real-time term on */
    int bdf_order;         /* 1 BE, 2 BDF2, 3 BDF3 */
    int alpha_pi_p_row;    /* 1: alpha_PI scales the pressure row too */
    double cfl_tau;
    double abs_tol[4];
} orc_problem;

void orc_flux_x(const double Q[5], double beta, double F[5]);
void orc_jacobian_x(const double Q[5], double beta, double A[25]);
void orc_eigen_x(const double Q[5], double beta, double lam[5], double R[25], double L[25]);
void orc_osher_x(const double QL[5], const double QR[5], double beta, double F[5]);
void orc_roe_x(const double QL[5], const double QR[5], double beta, double F[5]);
void orc_bassi_x(const double QL[5], const double QR[5], double beta, double F[5]);
void orc_bassi_star(const double WL[4], const double WR[4], double beta, double out[6]);
void orc_bassi_sample(const double WL[4], const double WR[4], double beta, double xi, double W[4]);
void orc_rotation(const double n[3], double Rm[25]);
void orc_face_flux(const double Qa[5], const double Qb[5], const double n[3], double beta,
                   int riemann, double F[5]);
double orc_limiter(double a, double b, double k);
void orc_bracket(const orc_problem *pb, const double *const q[4], const double *const rt[3],
                 const double *rho0, double *br[4]);
void orc_dtau(const orc_problem *pb, const double *const q[4], double *dtau);
double orc_realtime_dt(const orc_problem *pb, const double *const q[4], double cfl_t);
int orc_physical_step(const orc_problem *pb, double *q[4], const double *const hist[2][3],
                      double dt, double tol, int max_iters, int *iters, double R[4], double R0[4]);
int orc_pseudo_time_run(const orc_problem *pb, double *q[4], double tau_end, int max_iters, int *iters);

#ifdef __cplusplus
}
#endif
#endif
