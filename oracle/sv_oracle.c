/*
 * sv_oracle.c -- plain, slow, FP64 state-vector reference ("the oracle").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA path under paper_2503_19894_gb300/.
 *
 * What it computes (Section II-A of the paper, Eq. 1-3):
 *   - An n-qubit state is a length-2^n complex vector; qubit q is bit q of the
 *     amplitude index (Eq. 1 places U on qubit k as I^(n-k-1) (x) U (x) I^k,
 *     i.e. little-endian).
 *   - Applying a k-qubit gate U (2^k x 2^k) is 2^(n-k) independent matrix-vector
 *     products, one per group of 2^k amplitudes whose indices differ only in
 *     the target bits (Eq. 3).
 *
 * The group enumeration is deliberately the naive one: walk every index b in
 * [0, 2^n), skip it if any target bit is set, otherwise gather the 2^k members
 * b + sum_i bit_i(j) * 2^q[i].  No bit-insertion trick (Eq. 4) is used here.
 *
 * Matrix convention: row-major, complex128 interleaved (re, im); bit i of the
 * local row/column index corresponds to qubits[i] (caller's order).
 *
 * Parallelism: an OpenMP "parallel for" over b when compiled with -fopenmp;
 * every b is independent, so the result does not depend on the thread count.
 */
#include <complex.h>
#include <stdint.h>
#include <string.h>

#define ORC_MAX_K 10

/* Number of threads the OpenMP runtime will use (1 when built without it). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Apply one k-qubit gate in place (Eq. 3).
 *   psi    : 2^n complex amplitudes (interleaved re, im), modified in place
 *   n      : number of qubits
 *   qubits : k distinct qubit indices in [0, n), any order
 *   k      : gate size, 1 <= k <= ORC_MAX_K, k <= n
 *   mat    : 2^k x 2^k complex matrix, row-major
 * Returns 0 on success, -1 on a bad argument (nothing is modified then).
 */
int orc_apply_gate(double _Complex *psi, int n, const int *qubits, int k,
                   const double _Complex *mat)
{
    if (n < 1 || n > 40 || k < 1 || k > ORC_MAX_K || k > n)
        return -1;
    uint64_t tmask = 0;
    for (int i = 0; i < k; i++) {
        if (qubits[i] < 0 || qubits[i] >= n)
            return -1;
        uint64_t bit = (uint64_t)1 << qubits[i];
        if (tmask & bit)
            return -1; /* duplicate qubit */
        tmask |= bit;
    }
    const int64_t N = (int64_t)1 << n;
    const int K = 1 << k;

#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < N; b++) {
        if ((uint64_t)b & tmask)
            continue; /* not the base of a group */
        double _Complex x[1 << ORC_MAX_K];
        int64_t idx[1 << ORC_MAX_K];
        /* gather: member j has target bit q[i] equal to bit i of j */
        for (int j = 0; j < K; j++) {
            int64_t a = b;
            for (int i = 0; i < k; i++)
                if ((j >> i) & 1)
                    a += (int64_t)1 << qubits[i];
            idx[j] = a;
            x[j] = psi[a];
        }
        /* y = U x, then scatter back to the same addresses */
        for (int r = 0; r < K; r++) {
            double _Complex acc = 0.0;
            for (int c = 0; c < K; c++)
                acc += mat[(int64_t)r * K + c] * x[c];
            psi[idx[r]] = acc;
        }
    }
    return 0;
}

/*
 * Apply a list of gates one at a time, in order.
 *   n_gates  : number of gates
 *   ks       : gate sizes
 *   qubits   : all gates' qubit lists, concatenated (sum of ks entries)
 *   mats     : all gates' matrices, concatenated (sum of 4^k entries)
 * Returns 0, or -(g+1) for the first bad gate g (earlier gates are applied).
 */
int orc_apply_gates(double _Complex *psi, int n, int n_gates, const int *ks,
                    const int *qubits, const double _Complex *mats)
{
    int64_t qoff = 0, moff = 0;
    for (int g = 0; g < n_gates; g++) {
        int k = ks[g];
        if (orc_apply_gate(psi, n, qubits + qoff, k, mats + moff) != 0)
            return -(g + 1);
        qoff += k;
        moff += (int64_t)1 << (2 * k);
    }
    return 0;
}

/* <a|b> = sum_x conj(a_x) b_x over 2^n amplitudes, written in FP64. */
void orc_inner(const double _Complex *a, const double _Complex *b, int n,
               double *re, double *im)
{
    const int64_t N = (int64_t)1 << n;
    double sr = 0.0, si = 0.0;
#pragma omp parallel for reduction(+ : sr, si) schedule(static)
    for (int64_t x = 0; x < N; x++) {
        double _Complex p = conj(a[x]) * b[x];
        sr += creal(p);
        si += cimag(p);
    }
    *re = sr;
    *im = si;
}
