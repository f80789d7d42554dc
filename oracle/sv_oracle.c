/* CPU oracle: per-gate complex128 state-vector simulator -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain restatement of Sec. II.A of Doi & Horii: the state of n qubits is an array of 2^n
 * complex amplitudes, index bit k = qubit k (little-endian, Fig. 1-2).  A gate on qubits
 * (q0[, q1]) updates every group of 2^nq amplitudes whose indices differ only in those
 * bits (for one qubit: the pair i and i XOR 2^k, Fig. 2) by multiplying the group with the
 * gate's matrix.  One full pass over the array per gate; no blocking, no fusion.
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg load this library; the
 * CUDA library shares no code with it.
 *
 * Matrices are row-major 2^nq x 2^nq, interleaved (re, im) doubles, local index
 * b = bit(q0) + 2*bit(q1).  State arrays are interleaved (re, im) doubles.
 */
#include <complex.h>
#include <stdint.h>
#include <string.h>

typedef double _Complex cplx;

/* Index of group g with zero bits inserted at the positions in `pos` (ascending). */
static inline uint64_t insert_zeros(uint64_t g, const int *pos, int npos) {
    for (int j = 0; j < npos; ++j) {
        uint64_t low = g & ((1ull << pos[j]) - 1ull);
        g = ((g >> pos[j]) << (pos[j] + 1)) | low;
    }
    return g;
}

/* Apply one gate (Sec. II.A) in place. */
void oracle_apply_gate(double *state, int n, int nq, const int *q, const double *m) {
    cplx *a = (cplx *)state;
    int pos[2];
    pos[0] = q[0];
    if (nq == 2) {
        pos[0] = q[0] < q[1] ? q[0] : q[1];
        pos[1] = q[0] < q[1] ? q[1] : q[0];
    }
    const int dim = 1 << nq;
    cplx mat[16];
    for (int r = 0; r < dim; ++r)
        for (int c = 0; c < dim; ++c)
            mat[r * dim + c] = m[2 * (r * dim + c)] + I * m[2 * (r * dim + c) + 1];
    const int64_t groups = (int64_t)1 << (n - nq);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < groups; ++g) {
        uint64_t base = insert_zeros((uint64_t)g, pos, nq);
        uint64_t idx[4];
        cplx in[4];
        for (int b = 0; b < dim; ++b) {
            uint64_t i = base;
            if (b & 1) i |= 1ull << q[0];
            if (b & 2) i |= 1ull << q[1];
            idx[b] = i;
            in[b] = a[i];
        }
        for (int r = 0; r < dim; ++r) {
            cplx acc = 0;
            for (int c = 0; c < dim; ++c) acc += mat[r * dim + c] * in[c];
            a[idx[r]] = acc;
        }
    }
}

/* Apply a gate list: gate j has nq[j] qubits qs[2j], qs[2j+1] and matrix mats[32j ..]. */
void oracle_apply_circuit(double *state, int n, int64_t count, const int *nq, const int *qs,
                          const double *mats) {
    for (int64_t j = 0; j < count; ++j)
        oracle_apply_gate(state, n, nq[j], qs + 2 * j, mats + 32 * j);
}

/* |basis> : all amplitudes zero except index `basis` = 1 (Sec. IV.C initialisation). */
void oracle_init_basis(double *state, int n, uint64_t basis) {
    const int64_t len = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < len; ++i) {
        state[2 * i] = 0.0;
        state[2 * i + 1] = 0.0;
    }
    state[2 * basis] = 1.0;
}

/* Swap the contents of bit positions p and q of every index (a SWAP gate as a permutation). */
void oracle_swap_bits(double *state, int n, int p, int q) {
    cplx *a = (cplx *)state;
    const int64_t len = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < len; ++i) {
        uint64_t bp = ((uint64_t)i >> p) & 1ull, bq = ((uint64_t)i >> q) & 1ull;
        if (bp == 1 && bq == 0) {
            uint64_t j = (uint64_t)i ^ (1ull << p) ^ (1ull << q);
            cplx t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
}

/* Measurement probabilities |a_i|^2 (Sec. II.A). */
void oracle_probabilities(const double *state, int n, double *out) {
    const int64_t len = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < len; ++i)
        out[i] = state[2 * i] * state[2 * i] + state[2 * i + 1] * state[2 * i + 1];
}

/* Sum of |a_i|^2 over the whole state, accumulated in index order per thread block. */
double oracle_norm2(const double *state, int n) {
    const int64_t len = (int64_t)1 << n;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t i = 0; i < len; ++i) s += state[2 * i] * state[2 * i] + state[2 * i + 1] * state[2 * i + 1];
    return s;
}

/* <psi| P |psi> for the Pauli word P = i^{popc(x&z)} X^x Z^z (Y = iXZ on a qubit with both
 * bits):  sum_j conj(a_{j^x}) a_j (-1)^{popc(j&z)} i^{popc(x&z)}.  out = (re, im). */
void oracle_expval_pauli(const double *state, int n, uint64_t x, uint64_t z, double *out) {
    const cplx *a = (const cplx *)state;
    const int64_t len = (int64_t)1 << n;
    double sr = 0.0, si = 0.0;
#pragma omp parallel for reduction(+ : sr, si) schedule(static)
    for (int64_t j = 0; j < len; ++j) {
        cplx t = conj(a[(uint64_t)j ^ x]) * a[j];
        if (__builtin_popcountll((uint64_t)j & z) & 1) t = -t;
        sr += creal(t);
        si += cimag(t);
    }
    cplx s = sr + I * si;
    switch (__builtin_popcountll(x & z) & 3) {
        case 1: s *= I; break;
        case 2: s *= -1; break;
        case 3: s *= -I; break;
        default: break;
    }
    out[0] = creal(s);
    out[1] = cimag(s);
}

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the s-th output of the stream seeded with
 * `seed` is mix(seed + (s+1) * 0x9E3779B97F4A7C15).  Uniform double = top 53 bits * 2^-53. */
static inline uint64_t splitmix64_at(uint64_t seed, uint64_t s) {
    uint64_t z = seed + (s + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double oracle_uniform(uint64_t seed, uint64_t s) {
    return (double)(splitmix64_at(seed, s) >> 11) * 0x1.0p-53;
}

/* Inverse-CDF sampling: shot s returns the smallest i with cumsum_{k<=i} p_k > u_s * total,
 * where total = sum of all p_k.  Plain O(shots * 2^n) scan per shot would be too slow, so the
 * cumulative sums are formed once (sequentially, in index order) and searched by bisection. */
void oracle_sample(const double *probs, int n, int64_t shots, uint64_t seed, uint64_t *out,
                   double *cumsum_scratch) {
    const int64_t len = (int64_t)1 << n;
    double acc = 0.0;
    for (int64_t i = 0; i < len; ++i) {
        acc += probs[i];
        cumsum_scratch[i] = acc;
    }
    const double total = acc;
    for (int64_t s = 0; s < shots; ++s) {
        double t = oracle_uniform(seed, (uint64_t)s) * total;
        int64_t lo = 0, hi = len - 1; /* smallest i with cumsum[i] > t */
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (cumsum_scratch[mid] > t)
                hi = mid;
            else
                lo = mid + 1;
        }
        out[s] = (uint64_t)lo;
    }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
