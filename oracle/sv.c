/*
 * Oracle (test infrastructure only; never part of the product path).
 *
 * Plain complex128 state-vector simulator: the definition of an amplitude,
 * <b| U_circuit |0...0> (SM Sec. II), written out gate by gate.
 *
 * Conventions (the same ones the circuit generator documents):
 *   - qubit q is bit (n-1-q) of a basis index (qubit 0 is the most
 *     significant bit);
 *   - a gate matrix is row-major, row = output basis state;
 *   - a two-qubit gate on (a, b) with a < b uses the basis |q_a q_b>, i.e.
 *     matrix index 2*x_a + x_b.
 *
 * Storage: psi[2*i] = Re, psi[2*i+1] = Im of basis index i.
 * The parallel loops split the index range only; each output is computed
 * from the same inputs in the same order whatever the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static void apply_1q(double *psi, int n, int q, const double *m) {
    const int p = n - 1 - q;
    const int64_t half = (int64_t)1 << (n - 1);
    const int64_t low = ((int64_t)1 << p) - 1;
    const double m00r = m[0], m00i = m[1], m01r = m[2], m01i = m[3];
    const double m10r = m[4], m10i = m[5], m11r = m[6], m11i = m[7];
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < half; ++j) {
        int64_t i0 = ((j & ~low) << 1) | (j & low);
        int64_t i1 = i0 | ((int64_t)1 << p);
        double ar = psi[2 * i0], ai = psi[2 * i0 + 1];
        double br = psi[2 * i1], bi = psi[2 * i1 + 1];
        psi[2 * i0]     = m00r * ar - m00i * ai + m01r * br - m01i * bi;
        psi[2 * i0 + 1] = m00r * ai + m00i * ar + m01r * bi + m01i * br;
        psi[2 * i1]     = m10r * ar - m10i * ai + m11r * br - m11i * bi;
        psi[2 * i1 + 1] = m10r * ai + m10i * ar + m11r * bi + m11i * br;
    }
}

/* insert a zero bit at position p of x */
static inline int64_t ins0(int64_t x, int p) {
    int64_t low = ((int64_t)1 << p) - 1;
    return ((x & ~low) << 1) | (x & low);
}

static void apply_2q(double *psi, int n, int qa, int qb, const double *m) {
    const int pa = n - 1 - qa, pb = n - 1 - qb;  /* qa < qb  =>  pa > pb */
    const int64_t quarter = (int64_t)1 << (n - 2);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < quarter; ++j) {
        int64_t base = ins0(ins0(j, pb), pa);
        int64_t idx[4];
        idx[0] = base;                                   /* x_a=0 x_b=0 */
        idx[1] = base | ((int64_t)1 << pb);              /* x_a=0 x_b=1 */
        idx[2] = base | ((int64_t)1 << pa);              /* x_a=1 x_b=0 */
        idx[3] = base | ((int64_t)1 << pa) | ((int64_t)1 << pb);
        double in_r[4], in_i[4];
        for (int c = 0; c < 4; ++c) {
            in_r[c] = psi[2 * idx[c]];
            in_i[c] = psi[2 * idx[c] + 1];
        }
        for (int r = 0; r < 4; ++r) {
            double sr = 0.0, si = 0.0;
            for (int c = 0; c < 4; ++c) {
                double gr = m[2 * (4 * r + c)], gi = m[2 * (4 * r + c) + 1];
                sr += gr * in_r[c] - gi * in_i[c];
                si += gr * in_i[c] + gi * in_r[c];
            }
            psi[2 * idx[r]] = sr;
            psi[2 * idx[r] + 1] = si;
        }
    }
}

/* Evolve |0...0> through the gate list; psi must hold 2 * 2^n doubles. */
int oracle_sv_state(int n, int n_gates, const int32_t *q0, const int32_t *q1,
                    const double *mats, double *psi) {
    if (n < 1 || n > 40) return -1;
    const int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < 2 * dim; ++i) psi[i] = 0.0;
    psi[0] = 1.0;
    for (int g = 0; g < n_gates; ++g) {
        const double *m = mats + 32 * (int64_t)g;
        if (q1[g] < 0) {
            if (q0[g] < 0 || q0[g] >= n) return -2;
            apply_1q(psi, n, q0[g], m);
        } else {
            int a = q0[g], b = q1[g];
            if (a < 0 || b >= n || a >= b) return -3;
            apply_2q(psi, n, a, b, m);
        }
    }
    return 0;
}

/* Amplitudes of k bitstrings (bits[b*n + q] = value of qubit q). */
int oracle_sv_amplitudes(int n, int n_gates, const int32_t *q0, const int32_t *q1,
                         const double *mats, const uint8_t *bits, int64_t k,
                         double *amps) {
    const int64_t dim = (int64_t)1 << n;
    double *psi = (double *)malloc(sizeof(double) * 2 * (size_t)dim);
    if (!psi) return -10;
    int rc = oracle_sv_state(n, n_gates, q0, q1, mats, psi);
    if (rc == 0) {
        for (int64_t b = 0; b < k; ++b) {
            int64_t idx = 0;
            for (int q = 0; q < n; ++q) idx = (idx << 1) | (bits[b * n + q] & 1);
            amps[2 * b] = psi[2 * idx];
            amps[2 * b + 1] = psi[2 * idx + 1];
        }
    }
    free(psi);
    return rc;
}
