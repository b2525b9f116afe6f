/*
 * CPU oracle for exact state-vector / density-matrix simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or helper with the CUDA library, and never calls it.
 *
 * Plain, slow, obviously correct FP64.  Every function follows the passage
 * of the paper (QuEST, arXiv 1802.08032) named in its comment.
 *
 *   Amplitudes: double _Complex, index bit q = qubit q (Sec. II.B.1, Eq. 1).
 *   Density matrix of N qubits: the 2N-qubit vector rho'[j + 2^N k] = rho_jk
 *   (Sec. II.B.1, Eq. 2; row j in the low N bits, column k in the high N).
 *
 * The element-wise loops carry an OpenMP "parallel for": every iteration
 * writes amplitudes no other iteration reads, so results are bit-identical
 * to a serial run.  Reductions are serial, in index order, in long double
 * with Neumaier compensation.
 *
 * Parity status: every function is pinned by the CPU tests (dense Kronecker
 * matrices, Kraus sums, closed forms, invariants); none is "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef double _Complex cplx;

/* |0...0>  (Sec. III, initZeroState) */
void orc_init_zero(cplx *a, int nq) {
    const int64_t dim = (int64_t)1 << nq;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < dim; ++j) a[j] = 0.0;
    a[0] = 1.0;
}

/* |+>^n : every amplitude 2^(-n/2). */
void orc_init_plus(cplx *a, int nq) {
    const int64_t dim = (int64_t)1 << nq;
    const double v = 1.0 / sqrt((double)dim);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < dim; ++j) a[j] = v;
}

/*
 * Single-target gate G (row-major 2x2: g[0] g[1] / g[2] g[3]) on qubit q of
 * an nq-qubit vector, restricted to indices whose bits in ctrl_mask are all 1
 * (Eq. 1 and its multi-control generalisation, Sec. II.B.1):
 *   for i in [0, 2^(nq-1)):  n_i = floor(i / 2^q) 2^(q+1) + (i mod 2^q)
 *   (a[n_i], a[n_i + 2^q]) <- G (a[n_i], a[n_i + 2^q])
 */
void orc_apply_gate(cplx *a, int nq, int q, uint64_t ctrl_mask, const cplx *g) {
    const int64_t half = (int64_t)1 << (nq - 1);
    const int64_t stride = (int64_t)1 << q;
    const cplx g00 = g[0], g01 = g[1], g10 = g[2], g11 = g[3];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < half; ++i) {
        const int64_t ni = (i / stride) * 2 * stride + (i % stride);
        if (((uint64_t)ni & ctrl_mask) != ctrl_mask) continue;
        const cplx x = a[ni], y = a[ni + stride];
        a[ni] = g00 * x + g01 * y;
        a[ni + stride] = g10 * x + g11 * y;
    }
}

/* Multi-controlled phase flip: every amplitude whose index has all bits of
 * ctrl_mask set changes sign (a diagonal gate; controlled-Z when two bits). */
void orc_phase_flip(cplx *a, int nq, uint64_t ctrl_mask) {
    const int64_t dim = (int64_t)1 << nq;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < dim; ++j)
        if (((uint64_t)j & ctrl_mask) == ctrl_mask) a[j] = -a[j];
}

/*
 * Gate on qubit q of an N-qubit density matrix held as a 2N-qubit vector
 * (Eq. 2): G_q rho G_q^dagger is enacted as G*_{q+N} G_q rho', i.e. G on bit
 * q (controls on their row bits), then conj(G) on bit q+N (controls on the
 * matching column bits).
 */
void orc_apply_dm_gate(cplx *rho, int N, int q, uint64_t ctrl_mask, const cplx *g) {
    cplx gc[4];
    for (int k = 0; k < 4; ++k) gc[k] = conj(g[k]);
    orc_apply_gate(rho, 2 * N, q, ctrl_mask, g);
    orc_apply_gate(rho, 2 * N, q + N, ctrl_mask << N, gc);
}

/* Density-matrix phase flip: rho -> P rho P with P the diagonal sign
 * operator; by Eq. 2 that is the flip on the row bits then on the column
 * bits (P is real, so P* = P). */
void orc_dm_phase_flip(cplx *rho, int N, uint64_t ctrl_mask) {
    orc_phase_flip(rho, 2 * N, ctrl_mask);
    orc_phase_flip(rho, 2 * N, ctrl_mask << N);
}

/*
 * Single-qubit channel in Kraus form on qubit q of an N-qubit density matrix:
 * rho -> sum_k K_k rho K_k^dagger.  For fixed values of every other row and
 * column bit, the 2x2 block M[r][c] = rho(row bit q = r, column bit q = c)
 * transforms as M <- sum_k K_k M K_k^dagger, which is what is computed here,
 * block by block.  (Used for the dephasing and depolarising noise of the
 * paper's abstract and Sec. II.B.1; the Kraus operators are built by the
 * caller.)  K holds nk row-major 2x2 matrices.
 */
void orc_apply_kraus(cplx *rho, int N, int q, int nk, const cplx *K) {
    const int64_t dim = (int64_t)1 << (2 * N);
    const int64_t rbit = (int64_t)1 << q, cbit = (int64_t)1 << (q + N);
#pragma omp parallel for schedule(static)
    for (int64_t base = 0; base < dim; ++base) {
        if (base & (rbit | cbit)) continue;   /* visit each block once */
        cplx M[2][2], out[2][2] = {{0, 0}, {0, 0}};
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c)
                M[r][c] = rho[base + r * rbit + c * cbit];
        for (int k = 0; k < nk; ++k) {
            const cplx *Kk = K + 4 * k;
            cplx KM[2][2];
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c)
                    KM[r][c] = Kk[2 * r + 0] * M[0][c] + Kk[2 * r + 1] * M[1][c];
            /* (K M K^dagger)[r][c] = sum_s (K M)[r][s] conj(K[c][s]) */
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c)
                    out[r][c] += KM[r][0] * conj(Kk[2 * c + 0]) + KM[r][1] * conj(Kk[2 * c + 1]);
        }
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c)
                rho[base + r * rbit + c * cbit] = out[r][c];
    }
}

/* Neumaier-compensated long double accumulator. */
typedef struct { long double s, c; } acc_t;
static void acc_add(acc_t *A, long double x) {
    long double t = A->s + x;
    if (fabsl(A->s) >= fabsl(x)) A->c += (A->s - t) + x;
    else A->c += (x - t) + A->s;
    A->s = t;
}
static double acc_get(const acc_t *A) { return (double)(A->s + A->c); }

static long double abs2(cplx z) {
    long double re = creal(z), im = cimag(z);
    return re * re + im * im;
}

/* Total probability of a state vector: sum_j |a_j|^2 (index order). */
double orc_total_prob_sv(const cplx *a, int nq) {
    acc_t A = {0, 0};
    const int64_t dim = (int64_t)1 << nq;
    for (int64_t j = 0; j < dim; ++j) acc_add(&A, abs2(a[j]));
    return acc_get(&A);
}

/* Probability that qubit q reads `outcome`: sum over j with bit q = outcome. */
double orc_prob_outcome_sv(const cplx *a, int nq, int q, int outcome) {
    acc_t A = {0, 0};
    const int64_t dim = (int64_t)1 << nq;
    for (int64_t j = 0; j < dim; ++j)
        if (((j >> q) & 1) == outcome) acc_add(&A, abs2(a[j]));
    return acc_get(&A);
}

/* Trace of a density matrix: sum_j Re rho_jj, rho_jj at index j + 2^N j. */
double orc_total_prob_dm(const cplx *rho, int N) {
    acc_t A = {0, 0};
    const int64_t d = (int64_t)1 << N;
    for (int64_t j = 0; j < d; ++j) acc_add(&A, creal(rho[j + d * j]));
    return acc_get(&A);
}

double orc_prob_outcome_dm(const cplx *rho, int N, int q, int outcome) {
    acc_t A = {0, 0};
    const int64_t d = (int64_t)1 << N;
    for (int64_t j = 0; j < d; ++j)
        if (((j >> q) & 1) == outcome) acc_add(&A, creal(rho[j + d * j]));
    return acc_get(&A);
}

/* Purity Tr(rho^2) = sum_jk rho_jk rho_kj = sum_n |rho'_n|^2 (rho Hermitian). */
double orc_purity_dm(const cplx *rho, int N) {
    return orc_total_prob_sv(rho, 2 * N);
}

/* Projective measurement of qubit q onto `outcome` with probability p > 0:
 * a_j <- 0 where bit q != outcome, else a_j / sqrt(p). */
void orc_collapse_sv(cplx *a, int nq, int q, int outcome, double p) {
    const int64_t dim = (int64_t)1 << nq;
    const double s = 1.0 / sqrt(p);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < dim; ++j)
        a[j] = (((j >> q) & 1) == outcome) ? a[j] * s : 0.0;
}

/* Density matrix: rho <- P rho P / p with P = |o><o| on qubit q, i.e. keep
 * entries whose row bit q and column bit q both equal `outcome`, divided by p. */
void orc_collapse_dm(cplx *rho, int N, int q, int outcome, double p) {
    const int64_t dim = (int64_t)1 << (2 * N);
    const double s = 1.0 / p;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < dim; ++n) {
        const int rb = (int)((n >> q) & 1), cb = (int)((n >> (q + N)) & 1);
        rho[n] = (rb == outcome && cb == outcome) ? rho[n] * s : 0.0;
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Host threads for the element-wise loops (thread-scaling runs); results do
 * not depend on it (each iteration writes amplitudes no other reads). */
void orc_set_num_threads(int t) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(t > 0 ? t : 1);
#else
    (void)t;
#endif
}

/*
 * m-target gate U (2^m x 2^m, row-major; bit k of the block index is qubit
 * t[k]) on the amplitudes whose bits in ctrl_mask are all 1: for every base
 * index with the target bits 0, the 2^m amplitudes a[base + sum_k bit_k(l)
 * 2^t[k]] (l = 0..2^m-1) are replaced by U times them.  This is Eq. 1 with
 * the pair replaced by a block of 2^m amplitudes (the paper's multi-qubit
 * generalisation, Sec. II.B.1).
 */
void orc_apply_multi(cplx *a, int nq, const int *t, int m, uint64_t ctrl_mask, const cplx *U) {
    const int64_t dim = (int64_t)1 << nq;
    const int64_t bs = (int64_t)1 << m;
    uint64_t tmask = 0;
    for (int k = 0; k < m; ++k) tmask |= (uint64_t)1 << t[k];
#pragma omp parallel for schedule(static)
    for (int64_t base = 0; base < dim; ++base) {
        if ((uint64_t)base & tmask) continue;
        if (((uint64_t)base & ctrl_mask) != ctrl_mask) continue;
        cplx v[64], w[64];
        int64_t idx[64];
        for (int64_t l = 0; l < bs; ++l) {
            int64_t off = 0;
            for (int k = 0; k < m; ++k)
                if ((l >> k) & 1) off += (int64_t)1 << t[k];
            idx[l] = base + off;
            v[l] = a[idx[l]];
        }
        for (int64_t r = 0; r < bs; ++r) {
            cplx s = 0;
            for (int64_t c = 0; c < bs; ++c) s += U[r * bs + c] * v[c];
            w[r] = s;
        }
        for (int64_t l = 0; l < bs; ++l) a[idx[l]] = w[l];
    }
}

/* Density matrix: U on the row bits t, then conj(U) on the column bits t+N
 * (Eq. 2; the paper states the rule holds for multi-qubit gates). */
void orc_apply_dm_multi(cplx *rho, int N, const int *t, int m, uint64_t ctrl_mask, const cplx *U) {
    const int64_t bs = (int64_t)1 << m;
    cplx Uc[64 * 64];
    int tc[8];
    for (int64_t e = 0; e < bs * bs; ++e) Uc[e] = conj(U[e]);
    for (int k = 0; k < m; ++k) tc[k] = t[k] + N;
    orc_apply_multi(rho, 2 * N, t, m, ctrl_mask, U);
    orc_apply_multi(rho, 2 * N, tc, m, ctrl_mask << N, Uc);
}
