/*
 * fdas_oracle.c -- FP64 CPU oracle for the FDAS correlation (TEST INFRASTRUCTURE ONLY).
 *
 * This file is a plain, slow and deliberately unoptimised statement of what the FDAS
 * hot path computes, used only by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline / reference legs of bench.py.  The GPU library never links, includes or
 * calls it, and it includes nothing from the GPU library.
 *
 * What is computed (Adamek, Dimoudi, Giles & Armour 2017, "Improved Acceleration of the
 * GPU Fourier Domain Acceleration Search Algorithm", Section 1, Eq. 2):
 *
 *     P[z][r] = | sum_{q=-h}^{h} A_{r+q} * conj(Hn_q(z)) |^2 ,   A_k = 0 for k outside [0,n)
 *
 * with h = m/2 (m = template length), and Hn the predicted Fourier response H of a
 * constant-frequency-derivative signal (Section 1, the correlation technique of Ransom,
 * Eikenberry & Middleditch 2002, cited there) normalised to unit L2 norm over the taps
 * actually used ("predicted, normalized Fourier response", Section 1).
 *
 * The response of a unit signal that starts at bin r_i and drifts z bins over the
 * observation, at bin offset q from its mean bin r_i + z/2, with the DFT sign of Eq. 3:
 *
 *     H_q(z) = int_0^1 exp(i*pi*(z*u^2 - (z + 2q)*u)) du
 *
 * Completing the square (z > 0):
 *     H_q(z) = exp(-i*pi*(z+2q)^2/(4z)) / sqrt(2z) * [F(t1) - F(t0)],
 *     t0 = -(z+2q)/sqrt(2z),  t1 = (z-2q)/sqrt(2z),  F(x) = C(x) + i S(x)
 * and H_q(-z) = conj(H_{-q}(z)),  H_q(0) = delta_{q,0} for integer q.
 *
 * F(x) = int_0^x exp(i*pi*t^2/2) dt (Fresnel integrals, DLMF 7.2.6-7.2.8) is evaluated by
 *   - the termwise-integrated power series of exp(i*pi*t^2/2) for |x| < 1.5 (DLMF 7.6.4-7.6.5),
 *   - F(x) = (1+i)/2 * (1 - erfc(w)), w = sqrt(pi)/2*(1-i)*x (DLMF 7.5 / 7.7), with erfc(w)
 *     from the Laplace continued fraction (DLMF 7.9.2), evaluated by the modified Lentz
 *     method, for |x| >= 1.5.
 *
 * z and q are integers everywhere in this file (the z grid is zstep * integer).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

/* ---- Fresnel integrals F(x) = C(x) + i S(x) ------------------------------------------ */

/* DLMF 7.6.4-7.6.5: exp(i pi t^2/2) = sum_n (i pi/2)^n t^{2n} / n!, integrated term by term:
 * F(x) = sum_n (i pi / 2)^n x^{2n+1} / (n! (2n+1)). */
static cplx fresnel_series(double x) {
    cplx power = x;                      /* (i pi x^2/2)^n x / n!  for n = 0 */
    cplx sum = x;
    const cplx ratio = I * (M_PI / 2.0) * x * x;
    for (int n = 1; n < 400; ++n) {
        power *= ratio / (double)n;
        cplx term = power / (double)(2 * n + 1);
        sum += term;
        if (cabs(term) <= 1e-18 * cabs(sum)) break;
    }
    return sum;
}

/* DLMF 7.9.2 (Re w > 0):
 *   sqrt(pi) * exp(w^2) * erfc(w) = 1/(w + (1/2)/(w + 1/(w + (3/2)/(w + 2/(w + ...)))))
 * i.e. the continued fraction b0 + a1/(b1 + a2/(b2 + ...)) with b_j = w and a_j = j/2 is the
 * reciprocal.  Modified Lentz evaluation (Lentz 1976; Thompson & Barnett 1986). */
static cplx erfc_cf(cplx w) {
    const double tiny = 1e-300;
    cplx f = w;                          /* b0 */
    if (cabs(f) == 0.0) f = tiny;
    cplx C = f, D = 0.0;
    for (int j = 1; j < 100000; ++j) {
        const double a = 0.5 * (double)j;
        D = w + a * D;
        if (cabs(D) == 0.0) D = tiny;
        C = w + a / C;
        if (cabs(C) == 0.0) C = tiny;
        D = 1.0 / D;
        cplx delta = C * D;
        f *= delta;
        if (cabs(delta - 1.0) < 1e-16) break;
    }
    return cexp(-w * w) / (sqrt(M_PI) * f);
}

cplx oracle_fresnel_c(double x) {
    const double ax = fabs(x);
    cplx F;
    if (ax < 1.5) {
        F = fresnel_series(ax);
    } else {
        /* DLMF 7.7 / 7.5: F(x) = (1+i)/2 * erf(sqrt(pi)/2 (1-i) x) */
        cplx w = (sqrt(M_PI) / 2.0) * (1.0 - I) * ax;
        F = (1.0 + I) / 2.0 * (1.0 - erfc_cf(w));
    }
    return x < 0 ? -F : F;               /* C and S are odd */
}

void oracle_fresnel(double x, double* c_out, double* s_out) {
    cplx F = oracle_fresnel_c(x);
    *c_out = creal(F);
    *s_out = cimag(F);
}

/* ---- Predicted response H_q(z) --------------------------------------------------------- */

/* H_q(z) for integer z > 0, integer q: the completed-square closed form above.  The phase
 * pi*(z+2q)^2/(4z) is reduced exactly in integers: (z+2q)^2 mod 8z. */
static cplx response_pos(int64_t z, int64_t q) {
    const int64_t b = z + 2 * q;
    const int64_t period = 8 * z;
    int64_t red = (b % period) * (b % period) % period;  /* b^2 mod 8z, exact */
    if (red < 0) red += period;
    const double phase = -M_PI * (double)red / (4.0 * (double)z);
    const double s2z = sqrt(2.0 * (double)z);
    const double t0 = -(double)(z + 2 * q) / s2z;
    const double t1 = (double)(z - 2 * q) / s2z;
    const cplx diff = oracle_fresnel_c(t1) - oracle_fresnel_c(t0);
    return cexp(I * phase) / s2z * diff;
}

cplx oracle_response_c(int64_t z, int64_t q) {
    if (z == 0) return q == 0 ? 1.0 : 0.0;
    if (z > 0) return response_pos(z, q);
    return conj(response_pos(-z, -q));
}

void oracle_response(int64_t z, int64_t q, double* re, double* im) {
    cplx H = oracle_response_c(z, q);
    *re = creal(H);
    *im = cimag(H);
}

/* Normalised taps Hn_q(z), q = -h..h, written interleaved (re, im) to out[2*(q+h)].
 * normalise = 0 returns the raw H_q(z). */
void oracle_template(int64_t z, int h, int normalise, double* out) {
    const int ntap = 2 * h + 1;
    double norm2 = 0.0;
    for (int j = 0; j < ntap; ++j) {
        cplx H = oracle_response_c(z, (int64_t)(j - h));
        out[2 * j] = creal(H);
        out[2 * j + 1] = cimag(H);
        norm2 += creal(H) * creal(H) + cimag(H) * cimag(H);
    }
    if (normalise) {
        const double s = 1.0 / sqrt(norm2);
        for (int j = 0; j < 2 * ntap; ++j) out[j] *= s;
    }
}

/* ---- The f-fdot power plane by direct sum (Eq. 2) --------------------------------------- */

/* One output cell: | sum_q A[r+q] conj(Hn_q) |^2, spectrum given as interleaved float32. */
static double cell(const float* spec, int64_t n, const double* taps, int h, int64_t r) {
    cplx acc = 0.0;
    for (int q = -h; q <= h; ++q) {
        const int64_t k = r + q;
        if (k < 0 || k >= n) continue;
        const cplx a = (double)spec[2 * k] + I * (double)spec[2 * k + 1];
        const cplx t = taps[2 * (q + h)] + I * taps[2 * (q + h) + 1];
        acc += a * conj(t);
    }
    return creal(acc) * creal(acc) + cimag(acc) * cimag(acc);
}

/* Rows z_idx in [row0, row1) of the plane, z = -zmax + z_idx*zstep; out is (row1-row0) x n. */
int oracle_plane_rows(const float* spec, int64_t n, int zmax, int zstep, int m,
                      int row0, int row1, double* out) {
    if (n < 1 || zstep < 1 || zmax < 0 || m < 2 || (m & 1) || row0 < 0 || row1 < row0) return -1;
    const int h = m / 2;
    for (int row = row0; row < row1; ++row) {
        const int64_t z = -(int64_t)zmax + (int64_t)row * zstep;
        double* taps = (double*)malloc(sizeof(double) * 2 * (2 * h + 1));
        if (!taps) return -2;
        oracle_template(z, h, 1, taps);
        double* dst = out + (int64_t)(row - row0) * n;
        #pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < n; ++r) dst[r] = cell(spec, n, taps, h, r);
        free(taps);
    }
    return 0;
}

/* Sampled cells: out[i] = P[z_idx[i]][r[i]]. */
int oracle_plane_samples(const float* spec, int64_t n, int zmax, int zstep, int m,
                         int64_t count, const int32_t* z_idx, const int64_t* r, double* out) {
    if (n < 1 || zstep < 1 || zmax < 0 || m < 2 || (m & 1) || count < 0) return -1;
    const int h = m / 2;
    const int Z = 2 * (zmax / zstep) + 1;
    double* taps = (double*)malloc(sizeof(double) * 2 * (2 * h + 1) * (size_t)Z);
    char* have = (char*)calloc((size_t)Z, 1);
    if (!taps || !have) { free(taps); free(have); return -2; }
    for (int64_t i = 0; i < count; ++i) {
        if (z_idx[i] < 0 || z_idx[i] >= Z || r[i] < 0 || r[i] >= n) { free(taps); free(have); return -1; }
        have[z_idx[i]] = 1;
    }
    #pragma omp parallel for schedule(dynamic)
    for (int row = 0; row < Z; ++row)
        if (have[row])
            oracle_template(-(int64_t)zmax + (int64_t)row * zstep, h, 1,
                            taps + (size_t)row * 2 * (2 * h + 1));
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i)
        out[i] = cell(spec, n, taps + (size_t)z_idx[i] * 2 * (2 * h + 1), h, r[i]);
    free(taps);
    free(have);
    return 0;
}
