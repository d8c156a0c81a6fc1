/*
 * etics_oracle.h -- plain FP64 CPU oracle for the expansion force calculation
 * of Meiron, Li, Holley-Bockelmann & Spurzem, "Expansion Techniques for
 * Collisionless Stellar Dynamical Simulations" (ETICS).
 *
 * TEST INFRASTRUCTURE ONLY.  This file and etics_oracle.c are the slow,
 * obviously-correct reference that the CUDA library is checked against.
 * Nothing in the product path may include, link, load or call them; only the
 * tests, the package smoke check and the benchmark's CPU-baseline leg do.
 * They share no code, header, table or constant with the CUDA sources.
 *
 * Conventions (all functions):
 *   - G = 1, expansion centre at the origin, Hernquist scale length a = 1.
 *   - Positions are x,y,z triples (double[N][3]); masses double[N].
 *   - Real orthonormal spherical harmonics WITHOUT the Condon-Shortley phase:
 *       Y_l0  = N_l0 P_l^0(cos t)
 *       Y_lm  = sqrt2 N_lm P_l^m(cos t) cos(m phi)   (m > 0)
 *       Y_l-m = sqrt2 N_lm P_l^m(cos t) sin(m phi)   (m > 0)
 *     with P_l^m(t) = (1-t^2)^{m/2} d^m/dt^m P_l(t) (no (-1)^m) and
 *     N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).  So Y_11 = +sqrt(3/4pi) x/r.
 *     A harmonic index j = l*l + l + m, m in [-l, l].
 *   - SCF coefficients c[n][j], n in [0, n_max], j in [0, (l_max+1)^2).
 *   - Accelerations acc[N][3] = -grad(Phi); potentials pot[N].
 *
 * Every function returns 0 on success and a negative value on bad arguments.
 */
#ifndef ETICS_ORACLE_H
#define ETICS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Hernquist-Ostriker radial potential basis function (Sec. 2.5, HO92 basis):
 * phi = -r^l (1+r)^-(2l+1) C_n^(2l+3/2)(xi), xi = (r-1)/(r+1); dphi = d phi/dr. */
int etics_ref_phi_nl(int n, int l, double r, double *phi, double *dphi);

/* Normalisation J_nl = int_0^inf rho_nl(r) phi_nl(r) r^2 dr of the same basis. */
double etics_ref_jnl(int n, int l);

/* Real orthonormal Y_lm(theta, phi) of the direction (x,y,z) for all
 * l <= l_max, written to Y[l*l+l+m].  At the origin theta = phi = 0. */
int etics_ref_ylm(int l_max, double x, double y, double z, double *Y);

/* SCF coefficients (Sec. 2.4 eq. 18, Sec. 3.3 step 1):
 *   c[n][j] = (1/J_nl) sum_k m_k phi_nl(r_k) Y_j(theta_k, phi_k)
 * summed in fixed chunks of consecutive particles (each serially in particle
 * order; the chunk sums added in chunk order, the chunk length a function of
 * N alone), on all online cores; the result does not depend on the number
 * of threads. */
int etics_ref_scf_coeffs(const double *pos, const double *mass, long n_part,
                         int n_max, int l_max, double *coeffs);

/* SCF field at arbitrary points (Sec. 2.4 eq. 18, Sec. 3.3 step 2):
 *   Phi = sum c[n][j] phi_nl(r) Y_j,   acc = -grad Phi.
 * acc or pot may be NULL.  nthreads <= 0 uses all online cores. */
int etics_ref_scf_field(const double *pos, long n_part, int n_max, int l_max,
                        const double *coeffs, double *acc, double *pot,
                        int nthreads);

/* MEX field at the particles themselves (Sec. 2.4 eqs. 15-17, Sec. 2.2):
 * particles ordered by r^2 = (x*x + y*y) + z*z in FP64, ties by index;
 * q_lm(i) sums the particles strictly before i, p_lm(i) strictly after.
 * order (nullable) receives the sorted particle indices. */
int etics_ref_mex_field(const double *pos, const double *mass, long n_part,
                        int l_max, double *acc, double *pot, long *order);
/* The same with a thread count (<= 0: all online cores); the cumulative sums
 * stay serial, the per-particle moments and field terms run over threads, and
 * the result is bitwise the same for every thread count. */
int etics_ref_mex_field_t(const double *pos, const double *mass, long n_part,
                          int l_max, double *acc, double *pot, long *order, int nthreads);

/* The same three SCF functions for a chosen radial basis (Sec. 2.5):
 * basis 0 = Hernquist-Ostriker (as above), basis 1 = Clutton-Brock (the
 * Plummer model as zeroth term):
 *   phi_nl = -r^l (1+r^2)^-(l+1/2) C_n^(l+1)(xi),  xi = (r^2-1)/(r^2+1). */
int etics_ref_phi_nl_b(int basis, int n, int l, double r, double *phi, double *dphi);
double etics_ref_jnl_b(int basis, int n, int l);
int etics_ref_scf_coeffs_b(int basis, const double *pos, const double *mass, long n_part,
                           int n_max, int l_max, double *coeffs);
/* ... with a thread count (<= 0: all online cores; the result is bitwise the
 * same for every thread count). */
int etics_ref_scf_coeffs_bt(int basis, const double *pos, const double *mass, long n_part,
                            int n_max, int l_max, double *coeffs, int nthreads);
int etics_ref_scf_field_b(int basis, const double *pos, long n_part, int n_max, int l_max,
                          const double *coeffs, double *acc, double *pot, int nthreads);

/* Direct summation (Sec. 2.1 eq. 4), unsoftened, self term excluded. */
int etics_ref_direct(const double *pos, const double *mass, long n_part,
                     double *acc, double *pot, int nthreads);

/* One kick-drift-kick leapfrog step (Sec. 3.4, Sec. 5.4):
 *   v += dt/2 a(x);  x += dt v;  a = force(x);  v += dt/2 a.
 * acc holds a(x) on entry and a(x + dt v) on exit; pot receives the new
 * potential.  method 0 = SCF, 1 = MEX.  coeffs (nullable, SCF only)
 * receives the coefficients of the new positions. */
int etics_ref_leapfrog_step(double *pos, double *vel, const double *mass,
                            double *acc, double *pot, long n_part, double dt,
                            int method, int n_max, int l_max, double *coeffs,
                            int nthreads);

/* Number of worker threads the field loops use for nthreads <= 0. */
int etics_ref_default_threads(void);

#ifdef __cplusplus
}
#endif
#endif
