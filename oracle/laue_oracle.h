/*
 * laue_oracle.h — FP64 CPU oracle for the LaueOT Sinkhorn-EM hot path
 * (arXiv 2404.06478).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg call this library.  It shares no source,
 * header, table or helper with the CUDA path.
 *
 * Conventions (all arrays row-major, double precision):
 *   geom[]  : e[3], lam_min, lam_max, D, n_det, then per detector
 *             centre[3], normal[3], half_size  (7 doubles each, n_det <= 4)
 *   R[n*9]  : grain orientation (crystal -> lab), x[n*3] grain centre (mm)
 *   omega[t]: sample rotation angle (rad) about +y; Gamma_t = Ry(omega_t)
 *   planes  : w[m*3] unit crystal direction, d0[m] spacing of the base
 *             reflection, nharm[m] number of allowed harmonics n*g0
 *   spots   : observed p[i*3] sorted by angle, I_off[T+1]
 *   model   : J_off[T+1], grain[j], plane[j] (frozen list), centre c[j*3]
 *             and ray r[j*3] at the poses of the E-step
 *   potentials f[i], g[j] and dust potentials fd[nd], gd[nd] (nd = 1 in
 *             the global dustbin mode, T in the per-angle mode), in mm^2.
 */
#ifndef LAUE_ORACLE_H
#define LAUE_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

int orc_reflections(double a, int hmax, int centering, int cap,
                    double* w, double* d0, int* nharm, int* hkl0);

void orc_gamma(double omega, double G[9]);
void orc_cost_lengths(const double* geom, int n, const int* det, double* out);

long orc_forward(const double* geom, const double* w, const double* d0, const int* nharm, int M,
                 const double* R, const double* x, int N, const double* omega, int T,
                 long cap, int* J_off, int* grain, int* plane, double* ray4, double* spot3,
                 int* det, double* center3, signed char* vis_all, double* margin_all);

void orc_refresh(const double* geom, const double* w, const double* d0, const int* nharm,
                 const double* R, const double* x, const double* omega, int T,
                 const int* J_off, const int* grain, const int* plane,
                 double* ray4, double* center3);

double orc_pair_cost(const double* p, const double* c, const double* r, double D);
void orc_pair_costs(int n, const double* p, const double* c, const double* r, double D, double* out);

void orc_masses(int mode, double frac, int T, const int* I_off, const int* J_off,
                double* U, double* O);

int orc_sinkhorn(const double* Dj, int T, const int* I_off, const double* p,
                 const int* J_off, const double* c, const double* r,
                 double eps, double c_out, int mode, double frac, int n_iter, double tol,
                 int warm, double* f, double* g, double* fd, double* gd);

void orc_harvest(const double* Dj, int T, const int* I_off, const double* p,
                 const int* J_off, const double* c, const double* r,
                 double eps, double c_out, int mode, double frac,
                 const double* f, const double* g, const double* fd, const double* gd,
                 int* assign, double* margin, double* err, double* q, double* v);

int orc_mstep(const double* geom, const double* w, const double* omega, int T,
              const int* I_off, const double* p, const int* J_off,
              const int* grain, const int* plane, const int* det, int N,
              const double* cE, const double* rE,
              const double* f, const double* g, double eps,
              int n_newton, int n_mm, double tol_x, double tol_R, double hreg,
              double* R, double* x, double* stats);

double orc_eps_schedule(double eps_final, int n_em, int k);
double orc_eps_schedule_f(double eps_final, int n_em, int k, double factor);

int orc_em(const double* geom, const double* w, const double* d0, const int* nharm,
           const double* omega, int T, const int* I_off, const double* p,
           const int* J_off, const int* grain, const int* plane, const int* det, int N,
           double* R, double* x, double eps_final, int n_em, int n_sinkhorn,
           double c_out, int mode, double frac, int n_newton, int n_mm,
           double tol_x, double tol_R, double hreg, int mstep_kind,
           double* f, double* g, double* fd, double* gd, int* assign, double* margin);

int orc_single_fit(const double* geom, const double* w, const double* d0, const int* nharm, int M,
                   const double* omega, int T, const int* I_off, const double* p,
                   int S, const double* R0, const double* x0,
                   double eps_final, int k_max, double c_out,
                   int n_newton, int n_mm, double tol_x, double tol_R, double hreg,
                   double f_out, double anneal, int recut,
                   double* R_out, double* x_out, int* keep, double* unmatched);

int orc_spot_matrix(const double* geom, const double* w, const double* d0, const int* nharm, int M,
                    const double* omega, int T, const int* I_off, const double* p,
                    int Nc, const double* R, const double* x, double eps_s, double c_out,
                    double* Lbar);

int orc_spot_greedy(int I, int Nc, const double* Lbar, int kmax,
                    int* order, double* gain, double* F);

int orc_kstar(int K, const double* gain);

void orc_grain_objective(const double* geom, const double* w, const double* omega, int T,
                         const int* I_off, const double* p, const int* J_off,
                         const int* grain, const int* plane, const int* det, int N,
                         const double* cE, const double* rE,
                         const double* f, const double* g, double eps,
                         const double* R, const double* x, double* En);

void orc_grain_grad(const double* geom, const double* w, const double* omega, int T,
                    const int* I_off, const double* p, const int* J_off,
                    const int* grain, const int* plane, const int* det, int N,
                    const double* f, const double* g, double eps,
                    const double* R, const double* x, double* grad);

void orc_sym3_eig(const double A[9], double evals[3], double evecs[9]);
void orc_svd3(const double B[9], double U[9], double S[3], double V[9]);
int  orc_wahba(const double B[9], double R[9]);

void orc_grain_gn(const double* geom, const double* w, const double* omega, int T,
                  const int* I_off, const double* p, const int* J_off,
                  const int* grain, const int* plane, const int* det, int N,
                  const double* cE, const double* rE, const double* f, const double* g, double eps,
                  const double* R, const double* x, double* grad, double* H, double* value);
void orc_mstep_adjoint(const double* geom, const double* w, const double* omega, int T,
                       const int* I_off, const double* p, const int* J_off,
                       const int* grain, const int* plane, const int* det, int N,
                       const double* cE, const double* rE, const double* f, const double* g, double eps,
                       int n_steps, double lambda, double* R, double* x, double* step_norms);
int orc_sinkhorn_unbalanced(const double* Dj, int T, const int* I_off, const double* p,
                            const int* J_off, const double* c, const double* r,
                            double eps, double kappa, double lambda, int n_iter,
                            double* f, double* g);
void orc_harvest_unbalanced(const double* Dj, int T, const int* I_off, const double* p,
                            const int* J_off, const double* c, const double* r, double eps,
                            const double* f, const double* g, int* assign, double* margin,
                            double* rowmass, double* q);
int orc_set_threads(int n);
void orc_reciprocal_basis(double a, double b, double c, double alpha, double beta, double gamma, double B[9]);
int orc_reflections_hkl(const double B[9], const int* hkl, int n, int cap,
                        double* w, double* d0, int* nharm, int* hkl0);
void orc_knn(const double* Dj, int T, const int* I_off, const double* p, const int* J_off, const double* c,
             const double* r, int rho, int* nbr);
int orc_sinkhorn_sparse(const double* Dj, int T, const int* I_off, const double* p, const int* J_off,
                        const double* c, const double* r, double eps, double c_out, int mode, double frac,
                        int n_iter, int rho, double* f, double* g, double* fd, double* gd);
long orc_start_grid(long n_full, int sym, int k, double cube, long cap, double* R_out, double* x_out);

#ifdef __cplusplus
}
#endif
#endif
