// Focal-spot evaluation kernels (section "Centimeter-scale metalens at
// long-wave infrared"): the PSF line and its FWHM, the sample discs of
// radius 3 FWHM, the power inside them, the focusing efficiencies and the
// Strehl ratio of Eq. 9; the incident plane-wave intensity of a reference
// run; intensities of field samples and encircled power.  All small: one
// thread per wavelength for the scans and sums (n_lambda <= 8), one thread
// per sample for the elementwise work.  FP64 throughout (the lens-field
// transforms deliver FP64 fields).
#include "zda_internal.h"

namespace zda {
namespace {

__device__ __forceinline__ double intensity_at(const double2 *ex, const double2 *ey, size_t i, double n_top)
{
    const double2 a = ex[i], b = ey[i];
    return 0.5 * n_top * (a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
}

// PSF line: n_line points (x_i, 0), x_i = i x_max / (n_line - 1)
__global__ void k_eval_line_points(double *pts, int n_line, double x_max)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_line) return;
    pts[2 * i] = n_line > 1 ? x_max * i / (n_line - 1) : 0.0;
    pts[2 * i + 1] = 0.0;
}

// One thread per wavelength: the line's intensity (into line, if given), its
// value on the axis and the full width at half maximum (the first sample
// below half the axis value, linear interpolation between it and the one
// before; NaN if the line never falls below half)
__global__ void k_eval_fwhm(const double2 *field, int nl, int n_line, double x_max, double n_top, double *line,
                            double *fw, double *i0)
{
    const int l = threadIdx.x;
    if (l >= nl) return;
    const double2 *ex = field + (size_t)l * n_line, *ey = field + (size_t)(nl + l) * n_line;
    const double dx = n_line > 1 ? x_max / (n_line - 1) : 0.0;
    const double I0 = intensity_at(ex, ey, 0, n_top), half = 0.5 * I0;
    double w = nan(""), prev = I0;
    bool found = false;
    for (int i = 0; i < n_line; ++i) {
        const double I = intensity_at(ex, ey, i, n_top);
        if (line) line[(size_t)l * n_line + i] = I;
        if (!found && i > 0 && I < half) {
            const double x0 = dx * (i - 1), x1 = dx * i;
            w = 2.0 * (x0 + (half - prev) * (x1 - x0) / (I - prev));
            found = true;
        }
        prev = I;
    }
    fw[l] = w;
    i0[l] = I0;
}

// Disc samples of wavelength l: n_rad radii (i + 1/2) 3 FWHM_l / n_rad x n_ang
// angles 2 pi a / n_ang; point (l n_rad + i) n_ang + a.  A wavelength whose
// FWHM is not finite gets its samples on the axis (its results are NaN).
__global__ void k_eval_disc_points(const double *fw, int nl, int n_rad, int n_ang, double *pts)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int per = n_rad * n_ang;
    if (t >= nl * per) return;
    const int l = t / per, i = (t % per) / n_ang, a = t % n_ang;
    const double w = fw[l];
    const double rmax = isfinite(w) ? 3.0 * w : 0.0;
    const double r = (i + 0.5) * rmax / n_rad, ang = 2.0 * M_PI * a / n_ang;
    double s, c;
    sincos(ang, &s, &c);
    pts[2 * (size_t)t] = r * c;
    pts[2 * (size_t)t + 1] = r * s;
}

// One thread per wavelength: disc power (midpoint rule in r, mean over the
// angles) and the figures of merit; out[8 l ..] = fwhm, I(0), FE, relative FE,
// transmittance, Strehl ratio, disc power, transmitted power
__global__ void k_eval_finish(const double2 *field, int nl, int n_rad, int n_ang, const double *fw, const double *i0,
                              EvalScalars sc, double *out)
{
    const int l = threadIdx.x;
    if (l >= nl) return;
    const size_t npts = (size_t)nl * n_rad * n_ang;
    const double2 *ex = field + (size_t)l * npts, *ey = field + (size_t)(nl + l) * npts;
    const size_t base = (size_t)l * n_rad * n_ang;
    const double w = fw[l], rmax = 3.0 * w, dr = rmax / n_rad;
    double p_disc = 0.0;
    for (int i = 0; i < n_rad; ++i) {
        double m = 0.0;
        for (int a = 0; a < n_ang; ++a) m += intensity_at(ex, ey, base + (size_t)i * n_ang + a, sc.n_top);
        p_disc += (m / n_ang) * 2.0 * M_PI * ((i + 0.5) * dr);
    }
    p_disc *= dr;
    if (!isfinite(w)) p_disc = nan("");
    const double p_inc = sc.incident[l] * sc.area, pt = sc.p_trans[l], lam = sc.lambda[l];
    double *o = out + 8 * l;
    o[0] = w;
    o[1] = i0[l];
    o[2] = p_disc / p_inc;
    o[3] = p_disc / pt;
    o[4] = pt / p_inc;
    o[5] = i0[l] * lam * lam * sc.focal * sc.focal / (pt * sc.area);
    o[6] = p_disc;
    o[7] = pt;
}

// One thread per wavelength: the phi-mean of the monitor's E_r over the
// annulus [i0, i1) with the Bloch phase of each row removed, u; the incident
// plane-wave intensity (n/2) abs(2 u)^2 of the reference run
__global__ void k_incident_intensity(const float2 *mon, int nl, int nr, int nphi, int i0, int i1, double dphi,
                                     double n_sub, double *out)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    const size_t plane = (size_t)nr * nphi;
    const float2 *er = mon + (size_t)l * 2 * plane;        // [q][c][i][j], c = 0: E_r
    double ur = 0.0, ui = 0.0;
    for (int j = 0; j < nphi; ++j) {
        double s, c;
        sincos(-dphi * j, &s, &c);
        double sr = 0.0, si = 0.0;
        for (int i = i0; i < i1; ++i) {
            const float2 v = er[(size_t)i * nphi + j];
            sr += v.x;
            si += v.y;
        }
        ur += sr * c - si * s;
        ui += sr * s + si * c;
    }
    const double cnt = (double)(i1 - i0) * nphi;
    ur /= cnt;
    ui /= cnt;
    out[l] = 0.5 * n_sub * 4.0 * (ur * ur + ui * ui);
}

__global__ void k_field_intensity(const double2 *field, int nl, int n, double n_top, double *out)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)nl * n) return;
    out[t] = intensity_at(field, field + (size_t)nl * n, t, n_top);
}

// one thread per profile: P(rho_k) = sum of trapezoids of I(r) 2 pi r up to rho_k
__global__ void k_encircled_power(const double *r, const double *I, int n_prof, int n, double *out)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_prof) return;
    const double *f = I + (size_t)q * n;
    double *o = out + (size_t)q * n;
    double acc = 0.0, prev = f[0] * 2.0 * M_PI * r[0];
    o[0] = 0.0;
    for (int k = 1; k < n; ++k) {
        const double cur = f[k] * 2.0 * M_PI * r[k];
        acc += 0.5 * (cur + prev) * (r[k] - r[k - 1]);
        o[k] = acc;
        prev = cur;
    }
}

}  // namespace

void launch_eval_line_points(double *pts, int n_line, double x_max, cudaStream_t s)
{
    k_eval_line_points<<<(n_line + 127) / 128, 128, 0, s>>>(pts, n_line, x_max);
}

void launch_eval_fwhm(const double2 *field, int nl, int n_line, double x_max, double n_top, double *line, double *fw,
                      double *i0, cudaStream_t s)
{
    k_eval_fwhm<<<1, 32, 0, s>>>(field, nl, n_line, x_max, n_top, line, fw, i0);
}

void launch_eval_disc_points(const double *fw, int nl, int n_rad, int n_ang, double *pts, cudaStream_t s)
{
    const int n = nl * n_rad * n_ang;
    k_eval_disc_points<<<(n + 127) / 128, 128, 0, s>>>(fw, nl, n_rad, n_ang, pts);
}

void launch_eval_finish(const double2 *field, int nl, int n_rad, int n_ang, const double *fw, const double *i0,
                        const EvalScalars &sc, double *out, cudaStream_t s)
{
    k_eval_finish<<<1, 32, 0, s>>>(field, nl, n_rad, n_ang, fw, i0, sc, out);
}

void launch_incident_intensity(const float2 *mon, int nl, int nr, int nphi, int i0, int i1, double dphi, double n_sub,
                               double *out, cudaStream_t s)
{
    k_incident_intensity<<<(nl + 31) / 32, 32, 0, s>>>(mon, nl, nr, nphi, i0, i1, dphi, n_sub, out);
}

void launch_field_intensity(const double2 *field, int nl, int n, double n_top, double *out, cudaStream_t s)
{
    const size_t t = (size_t)nl * n;
    k_field_intensity<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(field, nl, n, n_top, out);
}

void launch_encircled_power(const double *r, const double *I, int n_prof, int n, double *out, cudaStream_t s)
{
    k_encircled_power<<<(n_prof + 31) / 32, 32, 0, s>>>(r, I, n_prof, n, out);
}

}  // namespace zda
