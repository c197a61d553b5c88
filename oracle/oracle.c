/*
 * oracle.c -- plain, slow, obviously correct complex128 state-vector simulator.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  It shares no code with the
 * CUDA path and must never be called by it.
 *
 * Conventions (Sec. II.A, Eq. STAT2): the state of L qubits is a vector of 2^L
 * complex amplitudes a_i; qubit q is bit q of the index i, qubit 0 the least
 * significant bit.  All arithmetic is IEEE double (the 13-15 digit arithmetic
 * Sec. III.A asks for).  Every gate is one full sweep over the index, done in
 * place, exactly as the update rules Eqs. NUM2-NUM8 describe; there is no
 * fusion, tiling, blocking or reordering of any kind.
 *
 * OpenMP (when compiled with -fopenmp) only splits the index loop of a sweep
 * over host threads; the pairs a sweep touches are disjoint, so the result does
 * not depend on the thread count.  Reductions use OpenMP's sum reduction.
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

/* Gate kinds; the order matches the table in inputs/circuits.py. */
enum {
    OR_H = 0, OR_X, OR_Y, OR_XB, OR_YB, OR_NOT, OR_R, OR_V, OR_SU2, OR_U, OR_SWAP
};

typedef struct {
    int32_t kind;
    int32_t t0;     /* target qubit */
    int32_t t1;     /* second target (SWAP only) */
    int32_t pad;
    uint64_t cmask; /* control qubits as a bit mask (all must be 1) */
    double p[8];    /* parameters */
} or_gate;

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* INITIAL STATE x (App. A): a_x = 1, every other amplitude 0. */
void or_set_basis(cplx *a, int n, uint64_t x)
{
    uint64_t D = 1ull << n;
    memset(a, 0, D * sizeof(cplx));
    a[x] = 1.0;
}

/*
 * The 2x2 matrix U of a single-qubit gate, row-major: a'0 = U00 a0 + U01 a1,
 * a'1 = U10 a0 + U11 a1 where a0 / a1 are the amplitudes whose target bit is
 * 0 / 1.  Returns 0 on success, -1 for a kind without a 2x2 matrix.
 */
int or_gate_matrix(int kind, const double *p, cplx U[4])
{
    const double s = 1.0 / sqrt(2.0);
    switch (kind) {
    case OR_H:  /* Eq. Hadamard / Eq. NUM2 */
        U[0] = s; U[1] = s; U[2] = s; U[3] = -s; return 0;
    case OR_X:  /* Eq. Xoperation / Eq. NUM3: a'0=(a0+i a1)/sqrt2, a'1=(a1+i a0)/sqrt2 */
        U[0] = s; U[1] = I * s; U[2] = I * s; U[3] = s; return 0;
    case OR_Y:  /* Eq. Yoperation / Eq. NUM4: a'0=(a0+a1)/sqrt2, a'1=(a1-a0)/sqrt2 */
        U[0] = s; U[1] = s; U[2] = -s; U[3] = s; return 0;
    case OR_XB: /* inverse of X (Sec. II.B): its conjugate transpose */
        U[0] = s; U[1] = -I * s; U[2] = -I * s; U[3] = s; return 0;
    case OR_YB: /* inverse of Y: its transpose (Y is real) */
        U[0] = s; U[1] = -s; U[2] = s; U[3] = s; return 0;
    case OR_NOT: /* the flip of CNOT / Toffoli (Eqs. NUM6, NUM8) */
        U[0] = 0; U[1] = 1; U[2] = 1; U[3] = 0; return 0;
    case OR_R:  /* Eq. singlephase / Eq. NUM5: a'1 = e^{i phi} a1 */
        U[0] = 1; U[1] = 0; U[2] = 0; U[3] = cexp(I * p[0]); return 0;
    case OR_V: { /* Eq. COMM4 / Eq. NUM7 */
        cplx e = cexp(I * p[0]);
        U[0] = 0.5 * (1 + e); U[1] = 0.5 * (1 - e);
        U[2] = 0.5 * (1 - e); U[3] = 0.5 * (1 + e);
        return 0;
    }
    case OR_SU2: /* unit quaternion (a,b,c,d) -> [[a+ib, c+id], [-c+id, a-ib]] */
        U[0] = p[0] + I * p[1]; U[1] = p[2] + I * p[3];
        U[2] = -p[2] + I * p[3]; U[3] = p[0] - I * p[1];
        return 0;
    case OR_U:
        for (int k = 0; k < 4; k++) U[k] = p[2 * k] + I * p[2 * k + 1];
        return 0;
    default:
        return -1;
    }
}

/*
 * Controlled single-qubit update.  For every index i whose target bit t is 0
 * and whose control bits (cmask) are all 1, the pair (a_i, a_{i+2^t}) is
 * replaced by U applied to it; all other amplitudes stay as they are.  With
 * cmask = 0 this is Eqs. NUM2-NUM5 for a general U; with one control it is
 * Eqs. NUM6-NUM7, with two controls Eq. NUM8.
 */
void or_apply_2x2(cplx *a, int n, int t, uint64_t cmask, const cplx U[4])
{
    const int64_t D = (int64_t)1 << n;
    const uint64_t bt = 1ull << t;
#pragma omp parallel for schedule(static)
    for (int64_t ii = 0; ii < D; ii++) {
        uint64_t i = (uint64_t)ii;
        if (i & bt) continue;
        if ((i & cmask) != cmask) continue;
        uint64_t j = i | bt;
        cplx a0 = a[i], a1 = a[j];
        a[i] = U[0] * a0 + U[1] * a1;
        a[j] = U[2] * a0 + U[3] * a1;
    }
}

/* Quantum SWAP gate of qubits q0, q1 (optionally controlled): exchange the
 * amplitudes a(..0_q1..1_q0..) and a(..1_q1..0_q0..). */
void or_apply_swap_gate(cplx *a, int n, int q0, int q1, uint64_t cmask)
{
    const int64_t D = (int64_t)1 << n;
    const uint64_t b0 = 1ull << q0, b1 = 1ull << q1;
#pragma omp parallel for schedule(static)
    for (int64_t ii = 0; ii < D; ii++) {
        uint64_t i = (uint64_t)ii;
        if (!(i & b0) || (i & b1)) continue;     /* visit bit q0 = 1, bit q1 = 0 */
        if ((i & cmask) != cmask) continue;
        uint64_t j = (i & ~b0) | b1;
        cplx tmp = a[i];
        a[i] = a[j];
        a[j] = tmp;
    }
}

/* Apply one gate.  Returns 0, or -1 for an unknown kind. */
int or_apply_gate(cplx *a, int n, const or_gate *g)
{
    if (g->kind == OR_SWAP) {
        or_apply_swap_gate(a, n, g->t0, g->t1, g->cmask);
        return 0;
    }
    cplx U[4];
    if (or_gate_matrix(g->kind, g->p, U) != 0) return -1;
    or_apply_2x2(a, n, g->t0, g->cmask, U);
    return 0;
}

/* Apply a gate list in order (the command loop of Sec. IV).  Returns the index
 * of the first bad gate plus one, or 0. */
int64_t or_run(cplx *a, int n, const or_gate *gs, int64_t ng)
{
    for (int64_t k = 0; k < ng; k++)
        if (or_apply_gate(a, n, &gs[k]) != 0) return k + 1;
    return 0;
}

/*
 * Dense k-qubit unitary U (2^k x 2^k, row-major) on qubits q[0..k-1]:
 * q[j] is bit j of the row/column index r of U.  For every index i whose k
 * selected bits are all zero, the 2^k amplitudes v_c = a_{i + sum_j c_j 2^q[j]}
 * are replaced by w_r = sum_c U_rc v_c.  This is the plain definition of a
 * gate acting on k qubits; k <= 12.
 */
int or_apply_dense(cplx *a, int n, int k, const int *q, const cplx *U)
{
    if (k < 1 || k > 12 || k > n) return -1;
    const int64_t D = (int64_t)1 << n;
    const int64_t K = (int64_t)1 << k;
    uint64_t qmask = 0;
    for (int j = 0; j < k; j++) qmask |= 1ull << q[j];
    uint64_t *off = (uint64_t *)malloc(K * sizeof(uint64_t));
    for (int64_t c = 0; c < K; c++) {
        uint64_t o = 0;
        for (int j = 0; j < k; j++)
            if ((c >> j) & 1) o |= 1ull << q[j];
        off[c] = o;
    }
#pragma omp parallel
    {
        cplx *v = (cplx *)malloc(K * sizeof(cplx));
        cplx *w = (cplx *)malloc(K * sizeof(cplx));
#pragma omp for schedule(static)
        for (int64_t ii = 0; ii < D; ii++) {
            uint64_t i = (uint64_t)ii;
            if (i & qmask) continue;
            for (int64_t c = 0; c < K; c++) v[c] = a[i | off[c]];
            for (int64_t r = 0; r < K; r++) {
                cplx s = 0;
                for (int64_t c = 0; c < K; c++) s += U[r * K + c] * v[c];
                w[r] = s;
            }
            for (int64_t r = 0; r < K; r++) a[i | off[r]] = w[r];
        }
        free(v);
        free(w);
    }
    free(off);
    return 0;
}

/*
 * Physical exchange of K pairs of bit positions (l[m], h[m]) of the amplitude
 * index: the data movement of the local/nonlocal qubit interchange,
 * Eq. onequbitchange (K = 1) and Eqs. twoqubitchange0-5 (K = 2), generalised to
 * K pairs as Sec. III.B describes.  out[pi(i)] = in[i] where pi(i) swaps bit
 * l[m] with bit h[m] of i for every m.  in and out must not overlap.
 */
void or_permute_bits(const cplx *in, cplx *out, int n, int K, const int *l, const int *h)
{
    const int64_t D = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t ii = 0; ii < D; ii++) {
        uint64_t i = (uint64_t)ii, j = i;
        for (int m = 0; m < K; m++) {
            uint64_t bl = (i >> l[m]) & 1, bh = (i >> h[m]) & 1;
            j &= ~((1ull << l[m]) | (1ull << h[m]));
            j |= (bl << h[m]) | (bh << l[m]);
        }
        out[j] = in[i];
    }
}

/* Eq. STAT1: sum_i |a_i|^2. */
double or_norm(const cplx *a, int n)
{
    const int64_t D = (int64_t)1 << n;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t i = 0; i < D; i++) {
        double re = creal(a[i]), im = cimag(a[i]);
        s += re * re + im * im;
    }
    return s;
}

/* Probability of observing basis state i: |a_i|^2 (Sec. II.A). */
void or_probs(const cplx *a, int n, double *out)
{
    const int64_t D = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < D; i++) {
        double re = creal(a[i]), im = cimag(a[i]);
        out[i] = re * re + im * im;
    }
}

/* Eq. Shor7: <Q_q> = sum_k |a_k|^2 k_q, the probability that qubit q is 1. */
void or_qubit_probs(const cplx *a, int n, double *out)
{
    const int64_t D = (int64_t)1 << n;
    for (int q = 0; q < n; q++) {
        const uint64_t bq = 1ull << q;
        double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
        for (int64_t ii = 0; ii < D; ii++) {
            uint64_t i = (uint64_t)ii;
            if (!(i & bq)) continue;
            double re = creal(a[i]), im = cimag(a[i]);
            s += re * re + im * im;
        }
        out[q] = s;
    }
}

/*
 * Basis-state sampling (Sec. V.B, the procedure that draws basis states |x>
 * with probability |<x|Phi>|^2).  For each uniform number u[j] in [0,1) the
 * sample is the smallest x with u[j] * total < P(0) + ... + P(x), the inverse
 * of the cumulative distribution; total is the norm, so an unnormalised state
 * samples its normalised distribution.  Plain linear scan per sample.
 */
void or_sample(const cplx *a, int n, const double *u, int64_t s, uint64_t *out)
{
    const int64_t D = (int64_t)1 << n;
    double total = or_norm(a, n);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < s; j++) {
        double target = u[j] * total, c = 0.0;
        int64_t x = D - 1;
        for (int64_t i = 0; i < D; i++) {
            double re = creal(a[i]), im = cimag(a[i]);
            c += re * re + im * im;
            if (target < c) { x = i; break; }
        }
        out[j] = (uint64_t)x;
    }
}
