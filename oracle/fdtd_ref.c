/*
 * ORACLE -- test infrastructure, not the product.
 *
 * Plain FP64 CPU reference of the cylindrical-coordinate FDTD time loop of
 * the zoned-discrete-axisymmetry method: the Bloch-reduced Maxwell equations
 * (Eqs. 1-5, section "Differentiable FDTD in cylindrical coordinates"),
 * discretised on a staggered Yee grid with leap-frog time stepping, with
 * stretched-coordinate (convolutional) PMLs in r and z, a soft current sheet
 * source, and running DFTs of E at a list of (signed) angular frequencies
 * (the multi-frequency DTFT of the hybrid time/frequency adjoint, same
 * section).  Only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark may load this code; the CUDA library never does.
 *
 * Readings of the paper that this file follows (all shared, in words, with
 * the CUDA path, never in code):
 *  - Fields are stored in "Bloch-periodic" form psi = u e^{i m phi}; Eq. 5's
 *    im/r terms then become plain phi-differences and the wedge wraps with
 *    psi(phi + tau) = e^{i m tau} psi(phi), tau = 2 pi / n.
 *  - Yee sites: E_r(i+1/2, j, k), E_phi(i, j+1/2, k), E_z(i, j, k+1/2),
 *    H_r(i, j+1/2, k+1/2), H_phi(i+1/2, j, k+1/2), H_z(i+1/2, j+1/2, k), with
 *    r_i = r_lo + i dr.  The (1/r) d/dr (r .) term of the z-curl takes r at
 *    both neighbours and 1/r at the centre.  PEC walls close the domain at
 *    r_lo, r_hi, z = 0 and z = nz dz (tangential E = 0 there).
 *  - CPML: each r- or z-derivative term D gets an auxiliary psi with
 *    psi <- b psi + c D and is replaced by D + psi (kappa = 1).  With
 *    rpml_metric == 0 the 1/r metric factors use the real radius and the
 *    whole (1/r) d/dr (r .) term is stretched.
 *  - rpml_metric == 1: inside the r-PML (radii whose CPML b is non-zero)
 *    the stretched radius r~ of the r-PML enters the metric factors
 *    (section "Differentiable FDTD": the stretched coordinate appears
 *    explicitly in the equations).  (1/r~) d/dr~ (r~ F) = (1/s_r) dF/dr +
 *    F / r~, so the z-curls split into a stretched derivative
 *    (F(i+1) - F(i)) / dr and a metric part X = (F(i+1) + F(i)) / 2 -+ dF/dphi;
 *    every metric part (and the phi-derivatives of the r-curls) is divided
 *    by r~ through 1/r~ = (1/r) (X + psi_m), psi_m <- bm psi_m + cm X, the
 *    same recursive convolution as the CPML with sigma_m = Omega / r
 *    (bm = cm = 0: r~ = r, only the derivative is stretched).  Outside the
 *    r-PML the updates are those of rpml_metric == 0 (the same in exact
 *    arithmetic there).
 *  - The source current J enters the E update as E += dt/eps (curl H - J)
 *    on the E_r and E_phi sites of one z-plane at t_{n+1/2}.
 *  - DFT: X(w) += E^{n+1} e^{i w t_{n+1}} dt after each E update.
 *  - Continuous axisymmetry (bor != 0, the axis zone): one phi cell, the
 *    fields are the m-th azimuthal harmonic u and every (1/r) d/dphi is
 *    exactly i m / r (Eq. 5 with the phi-dependence removed).  With r_lo = 0
 *    the axis r = 0 carries E_phi, E_z and H_r sites; for |m| = 1 E_z = 0 there
 *    and E_phi, H_r on the axis enter every other update multiplied by r = 0,
 *    so they are left at zero (they affect no other field, no DFT weight and
 *    no gradient: all carry the factor r).
 *
 * Array layout: every field is complex double [nr][nphi][nz] (z fastest).
 */
#include <complex.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int nr, nphi, nz, n_steps;
    double r_lo, dr, dz, dphi, dt;
    double bloch_re, bloch_im;            /* e^{i m tau} */
    const double *eps_r, *eps_p, *eps_z;  /* per E-site permittivity [nr][nphi][nz] */
    /* CPML b, c coefficients: r nodes (nr+1), r half nodes (nr),
       z nodes (nz+1), z half nodes (nz) */
    const double *br_n, *cr_n, *br_h, *cr_h, *bz_n, *cz_n, *bz_h, *cz_h;
    int src_k, n_src;
    const double *src_pat;    /* complex [n_src][2][nr][nphi]  (E_r, E_phi sites) */
    const double *src_time;   /* complex [n_steps][n_src], value at t_{n+1/2} */
    int n_freq;
    const double *twiddle;    /* complex [n_steps][n_freq] = e^{i w t_{n+1}} dt */
    int bor;                  /* 1: continuous axisymmetry, d/dphi -> i m */
    int m;                    /* azimuthal order for bor */
    int mon_k;                /* < 0: no monitor DFT */
    double *mon_dft;          /* complex [n_freq][2][nr][nphi] (E_r, E_phi) */
    int des_k0, des_nk;       /* des_nk == 0: no design-volume DFT */
    double *des_dft;          /* complex [n_freq][3][des_nk][nr][nphi] */
    double *state;            /* NULL, or complex [18][nr][nphi][nz] in/out */
    int nthreads;             /* 0: OpenMP default */
    int rpml_metric;          /* 1: stretched radius in the metric factors */
    const double *bm_n, *cm_n, *bm_h, *cm_h;   /* metric recursion, r nodes / half nodes */
} orc_problem;

#define NSTATE 18
enum { ER, EP, EZ, HR, HP, HZ,
       PS_HR_Z, PS_HP_Z, PS_HP_R, PS_HZ_R,     /* H-side CPML psi */
       PS_ER_Z, PS_EP_Z, PS_EP_R, PS_EZ_R,     /* E-side CPML psi */
       PS_HR_M, PS_HZ_M, PS_ER_M, PS_EZ_M };   /* metric psi (rpml_metric == 1) */

int orc_state_count(void) { return NSTATE; }

int orc_run(const orc_problem *p)
{
    const int nr = p->nr, np = p->nphi, nz = p->nz;
    const size_t ncell = (size_t)nr * np * nz;
    const double dr = p->dr, dz = p->dz, dphi = p->dphi, dt = p->dt;
    const cplx bloch = p->bloch_re + I * p->bloch_im;   /* psi(j + nphi) = bloch psi(j) */
    const cplx bloch_inv = conj(bloch);                 /* |bloch| = 1 */

#ifdef _OPENMP
    if (p->nthreads > 0) omp_set_num_threads(p->nthreads);
#endif
    cplx *f = (cplx *)calloc(NSTATE * ncell, sizeof(cplx));
    if (!f) return -3;
    if (p->state) memcpy(f, p->state, NSTATE * ncell * sizeof(cplx));
    cplx *Er = f + ER * ncell, *Ep = f + EP * ncell, *Ez = f + EZ * ncell;
    cplx *Hr = f + HR * ncell, *Hp = f + HP * ncell, *Hz = f + HZ * ncell;

    double *r_n = (double *)malloc((nr + 1) * sizeof(double));   /* r_i */
    double *r_h = (double *)malloc(nr * sizeof(double));         /* r_{i+1/2} */
    for (int i = 0; i <= nr; ++i) r_n[i] = p->r_lo + i * dr;
    for (int i = 0; i < nr; ++i) r_h[i] = p->r_lo + (i + 0.5) * dr;

#define AT(a, i, j, k) (a)[((size_t)(i) * np + (j)) * nz + (k)]

    const cplx *spat = (const cplx *)p->src_pat;
    const cplx *stim = (const cplx *)p->src_time;
    const cplx *tw = (const cplx *)p->twiddle;
    cplx *mon = (cplx *)p->mon_dft;
    cplx *des = (cplx *)p->des_dft;

    for (int n = 0; n < p->n_steps; ++n) {
        /* ---- H^{n+1/2} = H^{n-1/2} - dt curl E^n  (Eq. 3, mu = 1) ---- */
#pragma omp parallel for schedule(static)
        for (int i = 0; i < nr; ++i)
            for (int j = 0; j < np; ++j)
                for (int k = 0; k < nz; ++k) {
                    const int jp = (j + 1 < np) ? j + 1 : 0;
                    const cplx wrap = (j + 1 < np) ? 1.0 : bloch;
                    /* neighbours beyond the PEC walls are zero */
                    const cplx ez_jp = wrap * AT(Ez, i, jp, k);
                    const cplx er_jp = wrap * AT(Er, i, jp, k);
                    const cplx ep_kp = (k + 1 < nz) ? AT(Ep, i, j, k + 1) : 0.0;
                    const cplx er_kp = (k + 1 < nz) ? AT(Er, i, j, k + 1) : 0.0;
                    const cplx ez_ip = (i + 1 < nr) ? AT(Ez, i + 1, j, k) : 0.0;
                    const cplx ep_ip = (i + 1 < nr) ? AT(Ep, i + 1, j, k) : 0.0;

                    /* H_r at (r_i, phi_{j+1/2}, z_{k+1/2}); on the axis it stays 0 */
                    if (r_n[i] > 0.0) {
                        cplx d_phi = p->bor ? I * p->m * AT(Ez, i, j, k) / r_n[i]
                                            : (ez_jp - AT(Ez, i, j, k)) / (r_n[i] * dphi);
                        if (p->rpml_metric && p->br_n[i] != 0.0) {
                            const cplx X = p->bor ? I * p->m * AT(Ez, i, j, k) : (ez_jp - AT(Ez, i, j, k)) / dphi;
                            cplx *pm = &AT(f + PS_HR_M * ncell, i, j, k);
                            *pm = p->bm_n[i] * *pm + p->cm_n[i] * X;
                            d_phi = (X + *pm) / r_n[i];
                        }
                        cplx d_z = (ep_kp - AT(Ep, i, j, k)) / dz;
                        cplx *ps = &AT(f + PS_HR_Z * ncell, i, j, k);
                        *ps = p->bz_h[k] * *ps + p->cz_h[k] * d_z;
                        AT(Hr, i, j, k) -= dt * (d_phi - (d_z + *ps));
                    }
                    /* H_phi at (r_{i+1/2}, phi_j, z_{k+1/2}) */
                    {
                        cplx d_z = (er_kp - AT(Er, i, j, k)) / dz;
                        cplx d_r = (ez_ip - AT(Ez, i, j, k)) / dr;
                        cplx *psz = &AT(f + PS_HP_Z * ncell, i, j, k);
                        cplx *psr = &AT(f + PS_HP_R * ncell, i, j, k);
                        *psz = p->bz_h[k] * *psz + p->cz_h[k] * d_z;
                        *psr = p->br_h[i] * *psr + p->cr_h[i] * d_r;
                        AT(Hp, i, j, k) -= dt * ((d_z + *psz) - (d_r + *psr));
                    }
                    /* H_z at (r_{i+1/2}, phi_{j+1/2}, z_k) */
                    if (!(p->rpml_metric && p->br_h[i] != 0.0)) {
                        cplx d_r = (r_n[i + 1] * ep_ip - r_n[i] * AT(Ep, i, j, k)) / (r_h[i] * dr);
                        cplx d_phi = p->bor ? I * p->m * AT(Er, i, j, k) / r_h[i]
                                            : (er_jp - AT(Er, i, j, k)) / (r_h[i] * dphi);
                        cplx *ps = &AT(f + PS_HZ_R * ncell, i, j, k);
                        *ps = p->br_h[i] * *ps + p->cr_h[i] * d_r;
                        AT(Hz, i, j, k) -= dt * ((d_r + *ps) - d_phi);
                    } else {
                        const cplx d_r = (ep_ip - AT(Ep, i, j, k)) / dr;
                        const cplx X = 0.5 * (ep_ip + AT(Ep, i, j, k))
                                     - (p->bor ? I * p->m * AT(Er, i, j, k) : (er_jp - AT(Er, i, j, k)) / dphi);
                        cplx *ps = &AT(f + PS_HZ_R * ncell, i, j, k);
                        cplx *pm = &AT(f + PS_HZ_M * ncell, i, j, k);
                        *ps = p->br_h[i] * *ps + p->cr_h[i] * d_r;
                        *pm = p->bm_h[i] * *pm + p->cm_h[i] * X;
                        AT(Hz, i, j, k) -= dt * ((d_r + *ps) + (X + *pm) / r_h[i]);
                    }
                }

        /* ---- E^{n+1} = E^n + dt/eps (curl H^{n+1/2} - J^{n+1/2})  (Eq. 4) ---- */
#pragma omp parallel for schedule(static)
        for (int i = 0; i < nr; ++i)
            for (int j = 0; j < np; ++j)
                for (int k = 0; k < nz; ++k) {
                    const int jm = (j > 0) ? j - 1 : np - 1;
                    const cplx wrap = (j > 0) ? 1.0 : bloch_inv;
                    const cplx hz_jm = wrap * AT(Hz, i, jm, k);
                    const cplx hr_jm = wrap * AT(Hr, i, jm, k);
                    cplx jr = 0.0, jp = 0.0;
                    if (k == p->src_k)
                        for (int s = 0; s < p->n_src; ++s) {
                            const cplx a = stim[(size_t)n * p->n_src + s];
                            jr += a * spat[(((size_t)s * 2 + 0) * nr + i) * np + j];
                            jp += a * spat[(((size_t)s * 2 + 1) * nr + i) * np + j];
                        }

                    /* E_r at (r_{i+1/2}, phi_j, z_k); PEC at k = 0 */
                    if (k > 0) {
                        cplx d_phi = p->bor ? I * p->m * AT(Hz, i, j, k) / r_h[i]
                                            : (AT(Hz, i, j, k) - hz_jm) / (r_h[i] * dphi);
                        if (p->rpml_metric && p->br_h[i] != 0.0) {
                            const cplx X = p->bor ? I * p->m * AT(Hz, i, j, k) : (AT(Hz, i, j, k) - hz_jm) / dphi;
                            cplx *pm = &AT(f + PS_ER_M * ncell, i, j, k);
                            *pm = p->bm_h[i] * *pm + p->cm_h[i] * X;
                            d_phi = (X + *pm) / r_h[i];
                        }
                        cplx d_z = (AT(Hp, i, j, k) - AT(Hp, i, j, k - 1)) / dz;
                        cplx *ps = &AT(f + PS_ER_Z * ncell, i, j, k);
                        *ps = p->bz_n[k] * *ps + p->cz_n[k] * d_z;
                        AT(Er, i, j, k) += dt / AT(p->eps_r, i, j, k) * ((d_phi - (d_z + *ps)) - jr);
                    }
                    /* E_phi at (r_i, phi_{j+1/2}, z_k); PEC at i = 0 and k = 0 */
                    if (i > 0 && k > 0) {
                        cplx d_z = (AT(Hr, i, j, k) - AT(Hr, i, j, k - 1)) / dz;
                        cplx d_r = (AT(Hz, i, j, k) - AT(Hz, i - 1, j, k)) / dr;
                        cplx *psz = &AT(f + PS_EP_Z * ncell, i, j, k);
                        cplx *psr = &AT(f + PS_EP_R * ncell, i, j, k);
                        *psz = p->bz_n[k] * *psz + p->cz_n[k] * d_z;
                        *psr = p->br_n[i] * *psr + p->cr_n[i] * d_r;
                        AT(Ep, i, j, k) += dt / AT(p->eps_p, i, j, k) * (((d_z + *psz) - (d_r + *psr)) - jp);
                    }
                    /* E_z at (r_i, phi_j, z_{k+1/2}); PEC at i = 0 */
                    if (i > 0 && !(p->rpml_metric && p->br_n[i] != 0.0)) {
                        cplx d_r = (r_h[i] * AT(Hp, i, j, k) - r_h[i - 1] * AT(Hp, i - 1, j, k)) / (r_n[i] * dr);
                        cplx d_phi = p->bor ? I * p->m * AT(Hr, i, j, k) / r_n[i]
                                            : (AT(Hr, i, j, k) - hr_jm) / (r_n[i] * dphi);
                        cplx *ps = &AT(f + PS_EZ_R * ncell, i, j, k);
                        *ps = p->br_n[i] * *ps + p->cr_n[i] * d_r;
                        AT(Ez, i, j, k) += dt / AT(p->eps_z, i, j, k) * ((d_r + *ps) - d_phi);
                    } else if (i > 0) {
                        const cplx d_r = (AT(Hp, i, j, k) - AT(Hp, i - 1, j, k)) / dr;
                        const cplx X = 0.5 * (AT(Hp, i, j, k) + AT(Hp, i - 1, j, k))
                                     - (p->bor ? I * p->m * AT(Hr, i, j, k) : (AT(Hr, i, j, k) - hr_jm) / dphi);
                        cplx *ps = &AT(f + PS_EZ_R * ncell, i, j, k);
                        cplx *pm = &AT(f + PS_EZ_M * ncell, i, j, k);
                        *ps = p->br_n[i] * *ps + p->cr_n[i] * d_r;
                        *pm = p->bm_n[i] * *pm + p->cm_n[i] * X;
                        AT(Ez, i, j, k) += dt / AT(p->eps_z, i, j, k) * ((d_r + *ps) + (X + *pm) / r_n[i]);
                    }
                }

        /* ---- running DFT of E^{n+1} ---- */
        for (int q = 0; q < p->n_freq; ++q) {
            const cplx w = tw[(size_t)n * p->n_freq + q];
            if (p->mon_k >= 0 && mon) {
                const int k = p->mon_k;
                for (int i = 0; i < nr; ++i)
                    for (int j = 0; j < np; ++j) {
                        mon[(((size_t)q * 2 + 0) * nr + i) * np + j] += w * AT(Er, i, j, k);
                        mon[(((size_t)q * 2 + 1) * nr + i) * np + j] += w * AT(Ep, i, j, k);
                    }
            }
            if (p->des_nk > 0 && des) {
#pragma omp parallel for schedule(static)
                for (int kk = 0; kk < p->des_nk; ++kk) {
                    const int k = p->des_k0 + kk;
                    for (int i = 0; i < nr; ++i)
                        for (int j = 0; j < np; ++j) {
                            const size_t b = (size_t)i * np + j;
                            des[(((size_t)q * 3 + 0) * p->des_nk + kk) * nr * np + b] += w * AT(Er, i, j, k);
                            des[(((size_t)q * 3 + 1) * p->des_nk + kk) * nr * np + b] += w * AT(Ep, i, j, k);
                            des[(((size_t)q * 3 + 2) * p->des_nk + kk) * nr * np + b] += w * AT(Ez, i, j, k);
                        }
                }
            }
        }
    }
#undef AT
    if (p->state) memcpy(p->state, f, NSTATE * ncell * sizeof(cplx));
    free(r_n); free(r_h); free(f);
    return 0;
}
