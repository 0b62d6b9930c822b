/*
 * rcs_oracle.c -- complex128 CPU reference for random-circuit state construction,
 * sampling and linear XEB.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, includes or
 * calls this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg use it. It shares no code, header or table with the CUDA path.
 *
 * What it computes is the plain definition of the pipeline in Section 3.2 of the
 * paper (state construction -> measurement sampling -> linear XEB):
 *   psi = U_G ... U_2 U_1 |0...0>, every gate applied one at a time, in order,
 *   to a dense complex128 state of 2^n amplitudes (qubit q = bit q of the index);
 *   x_s = smallest i with C_i > u_s * T, where C_i = sum_{j<=i} |psi_j|^2 and
 *   T = C_{2^n - 1}, for uniforms u_s in [0,1) from Philox4x64-10;
 *   F = 2^n * mean_s p(x_s) - 1 with p(x) = |psi_x|^2 / T (linear XEB).
 * The paper defines none of the gate matrices; the readings used (principal
 * square roots of X, Y, W = (X+Y)/sqrt2; fSim(theta, phi) in the basis
 * |b_q1 b_q0>) are written out in orc_gate_matrix below.
 *
 * Sums over 2^n terms use Neumaier-compensated summation so that the CDF and the
 * norm carry an error of a few ulps of the total, independent of n.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { G_SQRT_X = 0, G_SQRT_Y = 1, G_SQRT_W = 2, G_FSIM = 3, G_U1 = 4, G_U2 = 5 };
enum { F_ADJOINT = 1 };

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- gate matrices */

/* Pauli-type matrix P for the square-root gates: X, Y, and W = (X + Y)/sqrt(2). */
static void pauli_of(int kind, cplx P[4]) {
    const cplx X[4] = {0, 1, 1, 0};
    const cplx Y[4] = {0, -I, I, 0};
    for (int e = 0; e < 4; ++e) {
        if (kind == G_SQRT_X) P[e] = X[e];
        else if (kind == G_SQRT_Y) P[e] = Y[e];
        else P[e] = (X[e] + Y[e]) / sqrt(2.0);
    }
}

/* Writes the 2^nq x 2^nq matrix of one gate (row-major complex128) into m and
 * returns nq, or -1 for an unknown kind.
 *   sqrtP  = ((1+i) I + (1-i) P) / 2, the principal square root of P (P^2 = I);
 *   fSim(theta, phi) = [[1,0,0,0],[0,cos t,-i sin t,0],[0,-i sin t,cos t,0],[0,0,0,e^{-i phi}]]
 *          with local index j = b(q0) + 2 b(q1);
 *   U1/U2 = the caller's matrix u (interleaved re/im, row-major).
 * flags & F_ADJOINT replaces the matrix by its conjugate transpose. */
int orc_gate_matrix(int kind, int flags, double theta, double phi, const double *u, cplx *m) {
    int nq;
    if (kind == G_SQRT_X || kind == G_SQRT_Y || kind == G_SQRT_W) {
        cplx P[4];
        pauli_of(kind, P);
        const cplx Id[4] = {1, 0, 0, 1};
        for (int e = 0; e < 4; ++e) m[e] = ((1 + I) * Id[e] + (1 - I) * P[e]) / 2.0;
        nq = 1;
    } else if (kind == G_FSIM) {
        for (int e = 0; e < 16; ++e) m[e] = 0;
        m[0 * 4 + 0] = 1;
        m[1 * 4 + 1] = cos(theta);
        m[1 * 4 + 2] = -I * sin(theta);
        m[2 * 4 + 1] = -I * sin(theta);
        m[2 * 4 + 2] = cos(theta);
        m[3 * 4 + 3] = cexp(-I * phi);
        nq = 2;
    } else if (kind == G_U1 || kind == G_U2) {
        nq = kind == G_U1 ? 1 : 2;
        int d = 1 << nq;
        for (int e = 0; e < d * d; ++e) m[e] = u[2 * e] + I * u[2 * e + 1];
    } else {
        return -1;
    }
    if (flags & F_ADJOINT) {
        int d = 1 << nq;
        cplx t[16];
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) t[r * d + c] = conj(m[c * d + r]);
        memcpy(m, t, sizeof(cplx) * d * d);
    }
    return nq;
}

/* ---------------------------------------------------------------- state update */

/* Applies the 2^k x 2^k matrix m to qubits t[0..k-1] of the n-qubit state psi:
 * for every assignment of the other n-k bits, the 2^k amplitudes
 * a_j = psi[base + sum_i bit_i(j) 2^{t_i}] are replaced by sum_l m[j][l] a_l.
 * Targets must be distinct and < n; k <= 10. */
void orc_apply_matrix(cplx *psi, int n, int k, const int *t, const cplx *m) {
    int d = 1 << k;
    int sorted[16];
    for (int i = 0; i < k; ++i) sorted[i] = t[i];
    for (int i = 1; i < k; ++i)
        for (int j = i; j > 0 && sorted[j - 1] > sorted[j]; --j) {
            int x = sorted[j];
            sorted[j] = sorted[j - 1];
            sorted[j - 1] = x;
        }
    int64_t nbase = (int64_t)1 << (n - k);
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nbase; ++b) {
        /* spread b over the non-target bits: insert a 0 at each target position */
        uint64_t base = (uint64_t)b;
        for (int i = 0; i < k; ++i) {
            uint64_t lowmask = ((uint64_t)1 << sorted[i]) - 1;
            base = ((base & ~lowmask) << 1) | (base & lowmask);
        }
        cplx a[1024], r[1024];
        uint64_t idx[1024];
        for (int j = 0; j < d; ++j) {
            uint64_t off = 0;
            for (int i = 0; i < k; ++i)
                if ((j >> i) & 1) off |= (uint64_t)1 << t[i];
            idx[j] = base | off;
            a[j] = psi[idx[j]];
        }
        for (int j = 0; j < d; ++j) {
            cplx s = 0;
            for (int l = 0; l < d; ++l) s += m[j * d + l] * a[l];
            r[j] = s;
        }
        for (int j = 0; j < d; ++j) psi[idx[j]] = r[j];
    }
}

/* |0...0> */
void orc_init_zero(cplx *psi, int n) {
    int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) psi[i] = 0;
    psi[0] = 1;
}

/* Applies gates g = 0..ngates-1 in order. Returns 0, or -(g+1) for a bad gate. */
int64_t orc_run(cplx *psi, int n, int64_t ngates, const int32_t *kind, const int32_t *flags,
                const int32_t *q0, const int32_t *q1, const double *theta, const double *phi,
                const double *const *u) {
    for (int64_t g = 0; g < ngates; ++g) {
        cplx m[16];
        int nq = orc_gate_matrix(kind[g], flags[g], theta[g], phi[g], u ? u[g] : NULL, m);
        if (nq < 0) return -(g + 1);
        int t[2] = {q0[g], q1[g]};
        for (int i = 0; i < nq; ++i)
            if (t[i] < 0 || t[i] >= n) return -(g + 1);
        if (nq == 2 && t[0] == t[1]) return -(g + 1);
        orc_apply_matrix(psi, n, nq, t, m);
    }
    return 0;
}

/* ---------------------------------------------------------------- reductions */

/* Neumaier-compensated sum of |psi_i|^2 over all 2^n amplitudes. */
double orc_norm2(const cplx *psi, int n) {
    int64_t N = (int64_t)1 << n;
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double x = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    return s + c;
}

/* ---------------------------------------------------------------- Philox4x64-10 */
/* Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten rounds of
 * two 64x64->128 multiplies with Weyl-sequence key bumps between rounds. */

static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL;

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

/* Uniform of shot s: word (s mod 4) of Philox4x64-10(counter = (s div 4, 0, 0, 0),
 * key = (seed, 0)), mapped to [0,1) as (x >> 11) * 2^-53. */
double orc_uniform(uint64_t seed, uint64_t s) {
    uint64_t ctr[4] = {s >> 2, 0, 0, 0}, key[2] = {seed, 0}, out[4];
    orc_philox4x64_10(ctr, key, out);
    return (double)(out[s & 3] >> 11) * 0x1.0p-53;
}

/* ---------------------------------------------------------------- sampling */

/* Draws shots s = first .. first+count-1: out[s - first] = smallest i with
 * C_i > u_s * T (strict, so zero-probability indices are never chosen).
 * C is built in full with a compensated running sum. Returns 0, or -1 when the
 * CDF does not fit in memory. */
int orc_sample(const cplx *psi, int n, uint64_t seed, uint64_t first, uint64_t count, uint64_t *out) {
    int64_t N = (int64_t)1 << n;
    double *C = (double *)malloc(sizeof(double) * (size_t)N);
    if (!C) return -1;
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double x = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
        C[i] = s + c;
    }
    double T = C[N - 1];
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < (int64_t)count; ++k) {
        double target = orc_uniform(seed, first + (uint64_t)k) * T;
        int64_t lo = 0, hi = N - 1; /* answer in [lo, hi]; C[N-1] = T > target */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (C[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        out[k] = (uint64_t)lo;
    }
    free(C);
    return 0;
}

/* ---------------------------------------------------------------- XEB */

/* Linear cross-entropy benchmark of the samples against psi:
 * F = 2^n * (1/N) sum_s |psi_{x_s}|^2 / T - 1, T = sum_i |psi_i|^2.
 * Returns NaN for an out-of-range sample or N = 0. */
double orc_xeb(const cplx *psi, int n, const uint64_t *x, int64_t count) {
    if (count <= 0) return NAN;
    double T = orc_norm2(psi, n);
    uint64_t N = (uint64_t)1 << n;
    double s = 0.0, c = 0.0;
    for (int64_t k = 0; k < count; ++k) {
        if (x[k] >= N) return NAN;
        cplx a = psi[x[k]];
        double p = (creal(a) * creal(a) + cimag(a) * cimag(a)) / T;
        double t = s + p;
        if (fabs(s) >= fabs(p)) c += (s - t) + p;
        else c += (p - t) + s;
        s = t;
    }
    return ldexp((s + c) / (double)count, n) - 1.0;
}
