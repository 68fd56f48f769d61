/*
 * Circuit-level CPU oracle: plain FP64 state-vector simulation of every
 * Hadamard-test circuit of the VQLS global cost, gate by gate, on n+1 qubits.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header or constant with the CUDA library.
 *
 * What it follows (D-VQLS, Sec. 2.1-2.3):
 *   - Eq. 1: C = 1 - |<b|A|x>|^2 / <x|A^dag A|x>, with A = sum_l c_l A_l (Eq. 3).
 *   - Each overlap is measured by a Hadamard test with a single ancilla
 *     measurement (Sec. 2.1, last paragraph; Sec. 2.2 after Eq. 4: separate
 *     circuits for the real and the imaginary part).
 *   - The local cost (Eq. 2, expanded in Eq. 4): the numerator overlaps
 *     <x| A_l^dag U_b P_j U_b^dag A_m |x> with P_j = (I + Z_j)/2 need the
 *     extra Hadamard tests gamma^j_lm = <x| A_l^dag U_b Z_j U_b^dag A_m |x>.
 *   - The circuit body of Sec. 2.3: ansatz V(theta), two controlled Pauli
 *     strings, ancilla preparation and measurement.  For delta_l the whole
 *     U = U_b^dag A_l V(theta) is controlled; the ansatz is the Ry + CZ-ring
 *     hardware-efficient ansatz.
 *
 * Conventions (the paper fixes none of them):
 *   - basis index i = sum_k i_k 2^k; system qubit k is bit k; the ancilla is
 *     bit n of the (n+1)-qubit register.
 *   - Pauli string from masks: sigma(x,z) = i^popc(x&z) X^x Z^z, i.e. Y where
 *     both bits are set; as a circuit, one controlled X / Y / Z per qubit.
 *   - Ry(t) = [[cos t/2, -sin t/2], [sin t/2, cos t/2]];  CZ = diag(1,1,1,-1).
 *   - Ansatz: Ry layer alpha[0..n), then d times { CZ ring ; Ry layer
 *     alpha[l*n .. l*n+n) }.  CZ ring = CZ(q,q+1) for q < n-1 plus CZ(n-1,0)
 *     when n >= 3.
 *   - U_b: H^(x)n when b = |+>^n (b_plus != 0); otherwise the phased
 *     Householder reflection e^{i phi}(I - 2 w w^dag / w^dag w),
 *     w = e^{i phi}|0> - b, e^{i phi} = b_0/|b_0| (1 when b_0 = 0), which maps
 *     |0> to b.
 *   - Real part: H(anc) . C-U . H(anc);  imaginary part: S^dag on the ancilla
 *     before the last H;  result = <Z_anc> = P(anc=0) - P(anc=1).
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

/* ---------------------------------------------------------------- gates */

static void gate_ry(cplx* psi, int nq, int q, double theta, int ctrl) {
    const double c = cos(0.5 * theta), s = sin(0.5 * theta);
    const size_t dim = (size_t)1 << nq, bit = (size_t)1 << q;
    const size_t cmask = ctrl >= 0 ? ((size_t)1 << ctrl) : 0;
    for (size_t i = 0; i < dim; ++i) {
        if ((i & bit) || (i & cmask) != cmask) continue;
        const cplx a = psi[i], b = psi[i | bit];
        psi[i] = c * a - s * b;
        psi[i | bit] = s * a + c * b;
    }
}

static void gate_h(cplx* psi, int nq, int q, int ctrl) {
    const double r = 1.0 / sqrt(2.0);
    const size_t dim = (size_t)1 << nq, bit = (size_t)1 << q;
    const size_t cmask = ctrl >= 0 ? ((size_t)1 << ctrl) : 0;
    for (size_t i = 0; i < dim; ++i) {
        if ((i & bit) || (i & cmask) != cmask) continue;
        const cplx a = psi[i], b = psi[i | bit];
        psi[i] = r * (a + b);
        psi[i | bit] = r * (a - b);
    }
}

/* Z on qubit q when all bits of `when` are set (CZ, CCZ, controlled Z). */
static void gate_phase_flip(cplx* psi, int nq, size_t when) {
    const size_t dim = (size_t)1 << nq;
    for (size_t i = 0; i < dim; ++i)
        if ((i & when) == when) psi[i] = -psi[i];
}

static void gate_cx(cplx* psi, int nq, int ctrl, int q) {
    const size_t dim = (size_t)1 << nq, bit = (size_t)1 << q, cm = (size_t)1 << ctrl;
    for (size_t i = 0; i < dim; ++i) {
        if ((i & bit) || !(i & cm)) continue;
        const cplx t = psi[i];
        psi[i] = psi[i | bit];
        psi[i | bit] = t;
    }
}

/* Y = [[0,-i],[i,0]]:  new[0] = -i old[1],  new[1] = i old[0]. */
static void gate_cy(cplx* psi, int nq, int ctrl, int q) {
    const size_t dim = (size_t)1 << nq, bit = (size_t)1 << q, cm = (size_t)1 << ctrl;
    for (size_t i = 0; i < dim; ++i) {
        if ((i & bit) || !(i & cm)) continue;
        const cplx a = psi[i], b = psi[i | bit];
        psi[i] = -I * b;
        psi[i | bit] = I * a;
    }
}

static void gate_sdg(cplx* psi, int nq, int q) {
    const size_t dim = (size_t)1 << nq, bit = (size_t)1 << q;
    for (size_t i = 0; i < dim; ++i)
        if (i & bit) psi[i] *= -I;
}

/* ------------------------------------------------------- circuit blocks */

/* The Ry + CZ-ring ansatz on system qubits 0..n-1, controlled by `ctrl`
 * (ctrl < 0: uncontrolled). */
static void ansatz(cplx* psi, int nq, int n, int d, const double* alpha, int ctrl) {
    const size_t cm = ctrl >= 0 ? ((size_t)1 << ctrl) : 0;
    for (int q = 0; q < n; ++q) gate_ry(psi, nq, q, alpha[q], ctrl);
    for (int l = 1; l <= d; ++l) {
        for (int q = 0; q + 1 < n; ++q)
            gate_phase_flip(psi, nq, cm | ((size_t)1 << q) | ((size_t)1 << (q + 1)));
        if (n >= 3) gate_phase_flip(psi, nq, cm | ((size_t)1 << (n - 1)) | (size_t)1);
        for (int q = 0; q < n; ++q) gate_ry(psi, nq, q, alpha[l * n + q], ctrl);
    }
}

/* Controlled Pauli string sigma(x,z), control = ancilla. */
static void controlled_pauli(cplx* psi, int nq, int n, int anc, uint32_t x, uint32_t z) {
    for (int q = 0; q < n; ++q) {
        const int xb = (x >> q) & 1, zb = (z >> q) & 1;
        if (xb && zb) gate_cy(psi, nq, anc, q);
        else if (xb) gate_cx(psi, nq, anc, q);
        else if (zb) gate_phase_flip(psi, nq, ((size_t)1 << anc) | ((size_t)1 << q));
    }
}

/* Controlled U_b^dag (see the header for U_b). */
static void controlled_ub_dag(cplx* psi, int nq, int n, int anc, const cplx* b, int b_plus) {
    if (b_plus) {
        for (int q = 0; q < n; ++q) gate_h(psi, nq, q, anc);
        return;
    }
    const size_t N = (size_t)1 << n;
    cplx ph = 1.0;
    if (cabs(b[0]) > 0.0) ph = b[0] / cabs(b[0]);
    cplx* w = (cplx*)malloc(N * sizeof(cplx));
    double ww = 0.0;
    for (size_t i = 0; i < N; ++i) {
        w[i] = (i == 0 ? ph : 0.0) - b[i];
        ww += creal(conj(w[i]) * w[i]);
    }
    cplx* v = psi + ((size_t)1 << anc); /* ancilla = 1 half (anc is the top bit) */
    if (ww > 0.0) {
        cplx wv = 0.0;
        for (size_t i = 0; i < N; ++i) wv += conj(w[i]) * v[i];
        const cplx f = 2.0 * wv / ww;
        for (size_t i = 0; i < N; ++i) v[i] -= f * w[i];
    }
    /* U_b^dag = e^{-i phi} (I - 2 w w^dag / w^dag w) */
    for (size_t i = 0; i < N; ++i) v[i] *= conj(ph);
    free(w);
}

/* Controlled U_b (see the header for U_b). */
static void controlled_ub(cplx* psi, int nq, int n, int anc, const cplx* b, int b_plus) {
    if (b_plus) {
        for (int q = 0; q < n; ++q) gate_h(psi, nq, q, anc);
        return;
    }
    const size_t N = (size_t)1 << n;
    cplx ph = 1.0;
    if (cabs(b[0]) > 0.0) ph = b[0] / cabs(b[0]);
    cplx* w = (cplx*)malloc(N * sizeof(cplx));
    double ww = 0.0;
    for (size_t i = 0; i < N; ++i) {
        w[i] = (i == 0 ? ph : 0.0) - b[i];
        ww += creal(conj(w[i]) * w[i]);
    }
    cplx* v = psi + ((size_t)1 << anc);
    if (ww > 0.0) {
        cplx wv = 0.0;
        for (size_t i = 0; i < N; ++i) wv += conj(w[i]) * v[i];
        const cplx f = 2.0 * wv / ww;
        for (size_t i = 0; i < N; ++i) v[i] -= f * w[i];
    }
    /* U_b = e^{i phi} (I - 2 w w^dag / w^dag w) */
    for (size_t i = 0; i < N; ++i) v[i] *= ph;
    free(w);
}

static double z_ancilla(const cplx* psi, int n) {
    const size_t N = (size_t)1 << n;
    double p0 = 0.0, p1 = 0.0;
    for (size_t i = 0; i < N; ++i) p0 += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    for (size_t i = N; i < 2 * N; ++i) p1 += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    return p0 - p1;
}

/* One Hadamard test for beta_lm = <psi| A_l^dag A_m |psi>, psi = V(alpha)|0>.
 * part = 0: real part, 1: imaginary part.  `buf` holds 2^(n+1) amplitudes. */
static double hadamard_beta(cplx* buf, int n, int d, const double* alpha,
                            uint32_t xl, uint32_t zl, uint32_t xm, uint32_t zm, int part) {
    const int nq = n + 1, anc = n;
    memset(buf, 0, sizeof(cplx) << nq);
    buf[0] = 1.0;
    gate_h(buf, nq, anc, -1);
    ansatz(buf, nq, n, d, alpha, -1);
    controlled_pauli(buf, nq, n, anc, xm, zm); /* A_m first, then A_l^dag = A_l */
    controlled_pauli(buf, nq, n, anc, xl, zl);
    if (part) gate_sdg(buf, nq, anc);
    gate_h(buf, nq, anc, -1);
    return z_ancilla(buf, n);
}

/* One Hadamard test for delta_l = <b| A_l |psi> = <0| U_b^dag A_l V |0>. */
static double hadamard_delta(cplx* buf, int n, int d, const double* alpha, const cplx* b,
                             int b_plus, uint32_t xl, uint32_t zl, int part) {
    const int nq = n + 1, anc = n;
    memset(buf, 0, sizeof(cplx) << nq);
    buf[0] = 1.0;
    gate_h(buf, nq, anc, -1);
    ansatz(buf, nq, n, d, alpha, anc);
    controlled_pauli(buf, nq, n, anc, xl, zl);
    controlled_ub_dag(buf, nq, n, anc, b, b_plus);
    if (part) gate_sdg(buf, nq, anc);
    gate_h(buf, nq, anc, -1);
    return z_ancilla(buf, n);
}

/* One Hadamard test for gamma^j_lm = <psi| A_l^dag U_b Z_j U_b^dag A_m |psi>,
 * the numerator overlaps of the local cost (Eq. 2, Eq. 4): controlled A_m,
 * controlled U_b^dag, controlled Z_j, controlled U_b, controlled A_l. */
static double hadamard_gamma(cplx* buf, int n, int d, const double* alpha, const cplx* b, int b_plus,
                             uint32_t xl, uint32_t zl, uint32_t xm, uint32_t zm, int j, int part) {
    const int nq = n + 1, anc = n;
    memset(buf, 0, sizeof(cplx) << nq);
    buf[0] = 1.0;
    gate_h(buf, nq, anc, -1);
    ansatz(buf, nq, n, d, alpha, -1);
    controlled_pauli(buf, nq, n, anc, xm, zm);
    controlled_ub_dag(buf, nq, n, anc, b, b_plus);
    gate_phase_flip(buf, nq, ((size_t)1 << anc) | ((size_t)1 << j));
    controlled_ub(buf, nq, n, anc, b, b_plus);
    controlled_pauli(buf, nq, n, anc, xl, zl);
    if (part) gate_sdg(buf, nq, anc);
    gate_h(buf, nq, anc, -1);
    return z_ancilla(buf, n);
}

/* ------------------------------------------------------------ C-ABI */

static int bad_args(int n, int d, int L) { return n < 1 || n > 20 || d < 0 || L < 0; }

/* Ansatz state V(alpha)|0> on n qubits, gate by gate (interleaved re,im). */
int oracle_ansatz_state(int n, int d, const double* alpha, double* psi_out) {
    if (bad_args(n, d, 0)) return 1;
    const size_t N = (size_t)1 << n;
    cplx* psi = (cplx*)calloc(N, sizeof(cplx));
    psi[0] = 1.0;
    ansatz(psi, n, n, d, alpha, -1);
    memcpy(psi_out, psi, N * sizeof(cplx));
    free(psi);
    return 0;
}

int oracle_hadamard_beta(int n, int d, const double* alpha, uint32_t xl, uint32_t zl,
                         uint32_t xm, uint32_t zm, double* re, double* im) {
    if (bad_args(n, d, 0)) return 1;
    cplx* buf = (cplx*)malloc(sizeof(cplx) << (n + 1));
    *re = hadamard_beta(buf, n, d, alpha, xl, zl, xm, zm, 0);
    *im = hadamard_beta(buf, n, d, alpha, xl, zl, xm, zm, 1);
    free(buf);
    return 0;
}

int oracle_hadamard_delta(int n, int d, const double* alpha, const double* b, int b_plus,
                          uint32_t xl, uint32_t zl, double* re, double* im) {
    if (bad_args(n, d, 0)) return 1;
    cplx* buf = (cplx*)malloc(sizeof(cplx) << (n + 1));
    *re = hadamard_delta(buf, n, d, alpha, (const cplx*)b, b_plus, xl, zl, 0);
    *im = hadamard_delta(buf, n, d, alpha, (const cplx*)b, b_plus, xl, zl, 1);
    free(buf);
    return 0;
}

/* All L*L + L terms at one angle vector, two circuits per term, OpenMP over
 * circuits.  beta: L*L complex (row l, column m), delta: L complex, both
 * interleaved.  nthreads <= 0: the OpenMP default.  Returns the number of
 * threads used. */
int oracle_circuit_terms(int n, int d, const double* alpha, const double* b, int b_plus, int L,
                         const uint32_t* x, const uint32_t* z, double* beta, double* delta,
                         int nthreads) {
    if (bad_args(n, d, L)) return -1;
    const long nterm = (long)L * L + L;
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        cplx* buf = (cplx*)malloc(sizeof(cplx) << (n + 1));
#ifdef _OPENMP
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 4)
#endif
        for (long t = 0; t < 2 * nterm; ++t) {
            const long term = t >> 1;
            const int part = (int)(t & 1);
            if (term < (long)L * L) {
                const int l = (int)(term / L), m = (int)(term % L);
                beta[2 * term + part] = hadamard_beta(buf, n, d, alpha, x[l], z[l], x[m], z[m], part);
            } else {
                const int l = (int)(term - (long)L * L);
                delta[2 * l + part] =
                    hadamard_delta(buf, n, d, alpha, (const cplx*)b, b_plus, x[l], z[l], part);
            }
        }
        free(buf);
    }
    return used;
}

/* All n L^2 numerator overlaps gamma^j_lm of the local cost at one angle
 * vector, two circuits each (real, imaginary), OpenMP over circuits.
 * gamma: n * L * L complex, index (j * L + l) * L + m, interleaved.
 * Returns the number of threads used. */
int oracle_circuit_local_terms(int n, int d, const double* alpha, const double* b, int b_plus, int L,
                               const uint32_t* x, const uint32_t* z, double* gamma, int nthreads) {
    if (bad_args(n, d, L)) return -1;
    const long nterm = (long)n * L * L;
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        cplx* buf = (cplx*)malloc(sizeof(cplx) << (n + 1));
#ifdef _OPENMP
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 4)
#endif
        for (long t = 0; t < 2 * nterm; ++t) {
            const long term = t >> 1;
            const int part = (int)(t & 1);
            const int j = (int)(term / ((long)L * L));
            const long r = term % ((long)L * L);
            const int l = (int)(r / L), m = (int)(r % L);
            gamma[2 * term + part] =
                hadamard_gamma(buf, n, d, alpha, (const cplx*)b, b_plus, x[l], z[l], x[m], z[m], j, part);
        }
        free(buf);
    }
    return used;
}
