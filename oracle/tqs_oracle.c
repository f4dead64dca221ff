/*
 * tqs_oracle.c -- plain, slow, FP64 CPU oracle for noisy Monte-Carlo state-vector
 * simulation with tree-based reuse of intermediate states (TQSim, Sec. 2.4 and 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file.  It shares no code with the CUDA path.
 *
 * Conventions (each restated from the paper or fixed by the reading it needs):
 *   - qubit q is bit q of the amplitude index (little-endian);
 *   - a two-qubit gate matrix acts on the local index k = bit(q0) + 2*bit(q1);
 *   - a depolarizing noise site follows every gate, on that gate's qubits
 *     (Sec. 2.4, Fig. 2b/3c); p is the probability of a non-identity Pauli,
 *     uniform over the 3 (one-qubit) or 15 (two-qubit) choices;
 *   - readout error flips each measured bit with probability pm (Sec. 4.3);
 *   - randomness is Philox4x32-10 (Salmon et al., SC'11) keyed by the seed with
 *     counter (id_lo, id_hi, index, domain); see the functions below.
 *
 * Parity status: the state-vector, noise, sampling and tree routines are pinned
 * by closed forms, invariants and the density-matrix oracle in the test suite.
 * The Philox stream is pinned word for word against PyTorch's ATen
 * Philox4x32-10 engine, an independent implementation, on 12,000 counter/key
 * pairs, and statistically (uniformity, avalanche).
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

/* Oracle-private gate codes (the Python wrapper maps gate names onto these). */
enum {
    G_H = 0, G_X, G_Y, G_Z, G_S, G_SDG, G_T, G_TDG, G_RX, G_RY, G_RZ, G_P,
    G_CX, G_CZ, G_CP, G_SWAP, G_U1, G_U2
};

enum { DOM_NOISE = 1, DOM_MEAS = 2, DOM_READ = 3, DOM_KRAUS = 4 };

/* ------------------------------------------------------------------------- */
/* Philox4x32-10: ten rounds of the 4x32 S-box with a Weyl key schedule.      */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint64_t id, uint32_t index, uint32_t domain, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), index, domain};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Threshold for an event of probability p on a uniform 32-bit word: floor(p * 2^32). */
static uint64_t threshold(double p)
{
    return (uint64_t)floor(p * 4294967296.0);
}

/* Noise at one site of one tree node: 0 = no error, else the Pauli index
 * 1..npaulis (npaulis = 3 for one-qubit sites, 15 for two-qubit sites). */
int orc_noise_draw(uint64_t seed, uint64_t node, uint32_t site, double p, int npaulis)
{
    uint32_t r[4];
    draw(seed, node, site, DOM_NOISE, r);
    if ((uint64_t)r[0] >= threshold(p))
        return 0;
    return 1 + (int)(((uint64_t)r[1] * (uint64_t)npaulis) >> 32);
}

/* Uniform double in [0,1) with 53 bits for the measurement of leaf `leaf`. */
double orc_measure_u(uint64_t seed, uint64_t leaf)
{
    uint32_t r[4];
    draw(seed, leaf, 0, DOM_MEAS, r);
    return ((double)(r[0] >> 5) * 67108864.0 + (double)(r[1] >> 6)) * (1.0 / 9007199254740992.0);
}

/* Readout flip mask of leaf `leaf` on n bits: bit q flips iff its draw is below floor(pm*2^32). */
uint64_t orc_readout_mask(uint64_t seed, uint64_t leaf, int n, double pm)
{
    uint64_t thr = threshold(pm), m = 0;
    for (int q = 0; q < n; q++) {
        uint32_t r[4];
        draw(seed, leaf, (uint32_t)q, DOM_READ, r);
        if ((uint64_t)r[0] < thr)
            m |= (uint64_t)1 << q;
    }
    return m;
}

/* ------------------------------------------------------------------------- */
/* Gate matrices (textbook definitions, Nielsen & Chuang conventions).        */
/* ------------------------------------------------------------------------- */
static int gate_arity(int kind)
{
    return (kind == G_CX || kind == G_CZ || kind == G_CP || kind == G_SWAP || kind == G_U2) ? 2 : 1;
}

/* Fills m (row-major, d x d with d = 2 or 4). `mat` holds interleaved (re, im)
 * entries for U1 (2x2) and U2 (4x4). */
static void gate_matrix(int kind, double th, const double *mat, cplx *m)
{
    const double r2 = 1.0 / sqrt(2.0);
    double c = cos(th / 2.0), s = sin(th / 2.0);
    int d = gate_arity(kind) == 1 ? 2 : 4;
    for (int i = 0; i < d * d; i++)
        m[i] = 0.0;
    switch (kind) {
    case G_H: m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2; break;
    case G_X: m[1] = 1.0; m[2] = 1.0; break;
    case G_Y: m[1] = -I; m[2] = I; break;
    case G_Z: m[0] = 1.0; m[3] = -1.0; break;
    case G_S: m[0] = 1.0; m[3] = I; break;
    case G_SDG: m[0] = 1.0; m[3] = -I; break;
    case G_T: m[0] = 1.0; m[3] = r2 + I * r2; break; /* e^{i pi/4} */
    case G_TDG: m[0] = 1.0; m[3] = r2 - I * r2; break;
    case G_RX: m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; break;
    case G_RY: m[0] = c; m[1] = -s; m[2] = s; m[3] = c; break;
    case G_RZ: m[0] = cexp(-I * th / 2.0); m[3] = cexp(I * th / 2.0); break;
    case G_P: m[0] = 1.0; m[3] = cexp(I * th); break;
    case G_U1:
        for (int i = 0; i < 4; i++)
            m[i] = mat[2 * i] + I * mat[2 * i + 1];
        break;
    /* two-qubit gates on the local index k = bit(q0) + 2 bit(q1) */
    case G_CX: /* control q0, target q1: |k=1> <-> |k=3> */
        m[0 * 4 + 0] = 1.0; m[2 * 4 + 2] = 1.0; m[1 * 4 + 3] = 1.0; m[3 * 4 + 1] = 1.0;
        break;
    case G_CZ:
        m[0] = 1.0; m[5] = 1.0; m[10] = 1.0; m[15] = -1.0;
        break;
    case G_CP:
        m[0] = 1.0; m[5] = 1.0; m[10] = 1.0; m[15] = cexp(I * th);
        break;
    case G_SWAP: /* |k=1> <-> |k=2> */
        m[0] = 1.0; m[1 * 4 + 2] = 1.0; m[2 * 4 + 1] = 1.0; m[15] = 1.0;
        break;
    case G_U2:
        for (int i = 0; i < 16; i++)
            m[i] = mat[2 * i] + I * mat[2 * i + 1];
        break;
    default: break;
    }
}

/* Exported so that tests can pin the matrices against textbook identities. */
void orc_gate_matrix(int kind, double theta, const double *mat, double *out)
{
    cplx m[16];
    gate_matrix(kind, theta, mat, m);
    int d = gate_arity(kind) == 1 ? 2 : 4;
    for (int i = 0; i < d * d; i++) {
        out[2 * i] = creal(m[i]);
        out[2 * i + 1] = cimag(m[i]);
    }
}

static void apply_1q(cplx *psi, int n, int q, const cplx *u)
{
    uint64_t dim = (uint64_t)1 << n, bit = (uint64_t)1 << q;
    for (uint64_t i = 0; i < dim; i++) {
        if (i & bit)
            continue;
        uint64_t j = i | bit;
        cplx a = psi[i], b = psi[j];
        psi[i] = u[0] * a + u[1] * b;
        psi[j] = u[2] * a + u[3] * b;
    }
}

static void apply_2q(cplx *psi, int n, int q0, int q1, const cplx *u)
{
    uint64_t dim = (uint64_t)1 << n, b0 = (uint64_t)1 << q0, b1 = (uint64_t)1 << q1;
    for (uint64_t i = 0; i < dim; i++) {
        if ((i & b0) || (i & b1))
            continue;
        uint64_t idx[4] = {i, i | b0, i | b1, i | b0 | b1};
        cplx v[4], w[4];
        for (int k = 0; k < 4; k++)
            v[k] = psi[idx[k]];
        for (int r = 0; r < 4; r++) {
            w[r] = 0.0;
            for (int k = 0; k < 4; k++)
                w[r] += u[r * 4 + k] * v[k];
        }
        for (int k = 0; k < 4; k++)
            psi[idx[k]] = w[k];
    }
}

typedef struct {
    int n, G;
    const int *kind, *q0, *q1;
    const double *theta, *mat; /* mat: 32 doubles per gate (only U1/U2 read them) */
} circuit;

static void apply_gate(cplx *psi, const circuit *c, int g)
{
    cplx u[16];
    gate_matrix(c->kind[g], c->theta[g], c->mat + 32 * (size_t)g, u);
    if (gate_arity(c->kind[g]) == 1)
        apply_1q(psi, c->n, c->q0[g], u);
    else
        apply_2q(psi, c->n, c->q0[g], c->q1[g], u);
}

/* Pauli index 0..3 = I, X, Y, Z on qubit q. */
static void apply_pauli(cplx *psi, int n, int q, int which)
{
    static const int kinds[4] = {-1, G_X, G_Y, G_Z};
    if (which == 0)
        return;
    cplx u[16];
    gate_matrix(kinds[which], 0.0, NULL, u);
    apply_1q(psi, n, q, u);
}

/* Depolarizing noise after gate g, drawn for tree node `node`. */
static void apply_noise(cplx *psi, const circuit *c, int g, uint64_t seed, uint64_t node,
                        double p1, double p2)
{
    if (gate_arity(c->kind[g]) == 1) {
        int t = orc_noise_draw(seed, node, (uint32_t)g, p1, 3);
        if (t)
            apply_pauli(psi, c->n, c->q0[g], t);
    } else {
        int t = orc_noise_draw(seed, node, (uint32_t)g, p2, 15);
        if (t) {
            apply_pauli(psi, c->n, c->q0[g], t >> 2); /* a on q0 */
            apply_pauli(psi, c->n, c->q1[g], t & 3);  /* b on q1 */
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Non-unitary channels by quantum trajectories (Sec. 4.3: thermal relaxation, */
/* amplitude damping and phase damping, each a set of Kraus operators).        */
/* ------------------------------------------------------------------------- */
/* Channel parameters, 6 doubles: kr[0] amplitude-damping gamma, kr[1]
 * phase-damping lambda, kr[2..3] the (gamma, lambda) pair that thermal
 * relaxation amounts to after a one-qubit gate, kr[4..5] the same after a
 * two-qubit gate (see orc_thermal_params).  A zero entry is no channel.
 *
 * After a gate and its depolarizing Pauli, each qubit of the gate (q0, then q1)
 * goes through, in this order: the thermal-relaxation damping, the
 * thermal-relaxation dephasing, amplitude damping, phase damping.  Each is one
 * trajectory step: with the normalised state psi and P1 = sum_{x_q = 1} |psi_x|^2,
 * the "jump" Kraus operator K1 is chosen with probability r * P1 (r = gamma or
 * lambda), else K0, and psi <- K psi / sqrt(probability of the choice):
 *   amplitude damping  K0 = diag(1, sqrt(1-gamma)),  K1 = sqrt(gamma) |0><1|
 *   phase damping      K0 = diag(1, sqrt(1-lambda)), K1 = sqrt(lambda) |1><1|
 * (Nielsen & Chuang, Sec. 8.3.5-8.3.6).  The choice draws u in [0, 1) with 53
 * bits from counter (node_lo, node_hi, 16 g + 8 i + c, 4), i = 0/1 the gate's
 * qubit and c = 0..3 the channel in the order above; K1 iff u < r * P1. */
static double kraus_u(uint64_t seed, uint64_t node, uint32_t index)
{
    uint32_t r[4];
    draw(seed, node, index, DOM_KRAUS, r);
    return ((double)(r[0] >> 5) * 67108864.0 + (double)(r[1] >> 6)) * (1.0 / 9007199254740992.0);
}

static void kraus_step(cplx *psi, int n, int q, double rate, int damping, double u)
{
    uint64_t dim = (uint64_t)1 << n, bit = (uint64_t)1 << q;
    double total = 0.0, one = 0.0;
    for (uint64_t x = 0; x < dim; x++) {
        double w = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
        total += w;
        if (x & bit)
            one += w;
    }
    double pj = rate * one / total;
    if (u < pj) {
        double sc = sqrt(rate / (pj * total));
        for (uint64_t x = 0; x < dim; x++) {
            if (!(x & bit))
                continue;
            if (damping) { /* sqrt(gamma) |0><1| */
                psi[x & ~bit] = sc * psi[x];
                psi[x] = 0.0;
            } else { /* sqrt(lambda) |1><1| */
                psi[x & ~bit] = 0.0;
                psi[x] = sc * psi[x];
            }
        }
    } else {
        double s0 = 1.0 / sqrt((1.0 - pj) * total), s1 = sqrt(1.0 - rate) * s0;
        for (uint64_t x = 0; x < dim; x++)
            psi[x] *= (x & bit) ? s1 : s0;
    }
}

static void apply_kraus(cplx *psi, const circuit *c, int g, uint64_t seed, uint64_t node, const double *kr)
{
    if (!kr)
        return;
    int two = gate_arity(c->kind[g]) == 2;
    double rate[4] = {kr[two ? 4 : 2], kr[two ? 5 : 3], kr[0], kr[1]};
    int damping[4] = {1, 0, 1, 0};
    for (int i = 0; i <= two; i++) {
        int q = i ? c->q1[g] : c->q0[g];
        for (int ch = 0; ch < 4; ch++)
            if (rate[ch] > 0.0)
                kraus_step(psi, c->n, q, rate[ch], damping[ch], kraus_u(seed, node, 16u * (uint32_t)g + 8u * (uint32_t)i + (uint32_t)ch));
    }
}

/* The (gamma, lambda) of amplitude damping followed by phase damping that make
 * up thermal relaxation towards |0> over a gate of duration t with times T1 and
 * T2 <= 2 T1: gamma = 1 - exp(-t/T1) (population decay) and
 * lambda = 1 - exp(t/T1 - 2t/T2), so that the coherence decays by
 * sqrt(1-gamma) sqrt(1-lambda) = exp(-t/T2).  Returns -1 when T2 > 2 T1. */
int orc_thermal_params(double t1, double t2, double t, double *gamma, double *lambda)
{
    if (t1 <= 0.0 || t2 <= 0.0 || t2 > 2.0 * t1 || t < 0.0)
        return -1;
    *gamma = 1.0 - exp(-t / t1);
    *lambda = 1.0 - exp(t / t1 - 2.0 * t / t2);
    if (*lambda < 0.0)
        *lambda = 0.0;
    return 0;
}

/* Measurement: the smallest y (in index order) whose running sum of |psi_y|^2
 * exceeds u * total; if rounding leaves none, the last y with nonzero weight. */
static uint64_t sample_index(const cplx *psi, int n, double u)
{
    uint64_t dim = (uint64_t)1 << n;
    double total = 0.0;
    for (uint64_t y = 0; y < dim; y++)
        total += creal(psi[y]) * creal(psi[y]) + cimag(psi[y]) * cimag(psi[y]);
    double target = u * total, acc = 0.0;
    uint64_t last = 0;
    for (uint64_t y = 0; y < dim; y++) {
        double w = creal(psi[y]) * creal(psi[y]) + cimag(psi[y]) * cimag(psi[y]);
        if (w > 0.0)
            last = y;
        acc += w;
        if (acc > target)
            return y;
    }
    return last;
}

/* ------------------------------------------------------------------------- */
/* Exported entry points                                                      */
/* ------------------------------------------------------------------------- */

/* Noiseless state after all gates, starting from |0...0>. psi_out: 2*2^n doubles. */
int orc_ideal_state(int n, int G, const int *kind, const int *q0, const int *q1,
                    const double *theta, const double *mat, double *psi_out)
{
    circuit c = {n, G, kind, q0, q1, theta, mat};
    uint64_t dim = (uint64_t)1 << n;
    cplx *psi = calloc(dim, sizeof(cplx));
    if (!psi)
        return -1;
    psi[0] = 1.0;
    for (int g = 0; g < G; g++)
        apply_gate(psi, &c, g);
    memcpy(psi_out, psi, dim * sizeof(cplx));
    free(psi);
    return 0;
}

/* Tree description (Sec. 3.1): L = k+1 levels, arity[0..k], split[0..L] gate
 * boundaries with split[0] = 0 and split[L] = G.  Level i holds
 * M_i = prod_{j<=i} arity[j] instances; instance m of level i has parent
 * m / arity[i].  With N shots, only leaves m < N are simulated, and a node of
 * level i exists iff m < ceil(N / prod_{j>i} arity[j]). */
typedef struct {
    int L;
    const uint64_t *arity;
    const int *split;
    uint64_t N;
    uint64_t below[64]; /* below[i] = prod_{j>i} arity[j] */
} tree;

static void tree_init(tree *t, int L, const uint64_t *arity, const int *split, uint64_t N)
{
    t->L = L;
    t->arity = arity;
    t->split = split;
    t->N = N;
    uint64_t r = 1;
    for (int i = L - 1; i >= 0; i--) {
        t->below[i] = r;
        r *= arity[i];
    }
}

static int node_exists(const tree *t, int level, uint64_t m)
{
    /* m < ceil(N / below) <=> m * below < N */
    return m * t->below[level] < t->N;
}

typedef struct {
    const circuit *c;
    const tree *t;
    uint64_t seed;
    double p1, p2, pm;
    uint64_t *counts;
    cplx **stack; /* one state per level */
    const double *kr; /* channel parameters (apply_kraus) or NULL */
} tree_run;

static void run_node(tree_run *R, int level, uint64_t m)
{
    const circuit *c = R->c;
    uint64_t dim = (uint64_t)1 << c->n;
    cplx *psi = R->stack[level];
    if (level == 0) {
        memset(psi, 0, dim * sizeof(cplx));
        psi[0] = 1.0;
    } else {
        memcpy(psi, R->stack[level - 1], dim * sizeof(cplx));
    }
    for (int g = R->t->split[level]; g < R->t->split[level + 1]; g++) {
        apply_gate(psi, c, g);
        apply_noise(psi, c, g, R->seed, m, R->p1, R->p2);
        apply_kraus(psi, c, g, R->seed, m, R->kr);
    }
    if (level == R->t->L - 1) {
        uint64_t y = sample_index(psi, c->n, orc_measure_u(R->seed, m));
        y ^= orc_readout_mask(R->seed, m, c->n, R->pm);
        R->counts[y] += 1;
        return;
    }
    uint64_t a = R->t->arity[level + 1];
    for (uint64_t j = 0; j < a; j++) {
        uint64_t child = m * a + j;
        if (node_exists(R->t, level + 1, child))
            run_node(R, level + 1, child);
    }
}

/* Noisy Monte-Carlo with tree reuse.  The baseline simulator is the one-level
 * tree (N).  counts: 2^n uint64, zeroed here.  Level-0 subtrees are independent
 * and run on `threads` OpenMP threads (0 = default), each with its own
 * histogram; the summed histogram does not depend on the thread count. */
int orc_run_tree_k(int n, int G, const int *kind, const int *q0, const int *q1,
                   const double *theta, const double *mat, double p1, double p2, double pm,
                   const double *kr, uint64_t N, uint64_t seed, int L, const uint64_t *arity,
                   const int *split, int threads, uint64_t *counts);

int orc_run_tree(int n, int G, const int *kind, const int *q0, const int *q1,
                 const double *theta, const double *mat, double p1, double p2, double pm,
                 uint64_t N, uint64_t seed, int L, const uint64_t *arity, const int *split,
                 int threads, uint64_t *counts)
{
    return orc_run_tree_k(n, G, kind, q0, q1, theta, mat, p1, p2, pm, NULL, N, seed, L, arity, split,
                          threads, counts);
}

/* As orc_run_tree, with the non-unitary channels of `kr` (apply_kraus; NULL = none). */
int orc_run_tree_k(int n, int G, const int *kind, const int *q0, const int *q1,
                   const double *theta, const double *mat, double p1, double p2, double pm,
                   const double *kr, uint64_t N, uint64_t seed, int L, const uint64_t *arity,
                   const int *split, int threads, uint64_t *counts)
{
    circuit c = {n, G, kind, q0, q1, theta, mat};
    tree t;
    tree_init(&t, L, arity, split, N);
    uint64_t dim = (uint64_t)1 << n;
    memset(counts, 0, dim * sizeof(uint64_t));
    uint64_t roots = (N + t.below[0] - 1) / t.below[0];
    int fail = 0;
#ifdef _OPENMP
    if (threads > 0)
        omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel
    {
        uint64_t *local = calloc(dim, sizeof(uint64_t));
        cplx **stack = calloc((size_t)L, sizeof(cplx *));
        int ok = local && stack;
        for (int i = 0; ok && i < L; i++) {
            stack[i] = malloc(dim * sizeof(cplx));
            ok = stack[i] != NULL;
        }
        if (!ok) {
#pragma omp atomic write
            fail = 1;
        } else {
            tree_run R = {&c, &t, seed, p1, p2, pm, local, stack, kr};
#pragma omp for schedule(dynamic, 1)
            for (int64_t m = 0; m < (int64_t)roots; m++)
                run_node(&R, 0, (uint64_t)m);
#pragma omp critical
            for (uint64_t y = 0; y < dim; y++)
                counts[y] += local[y];
        }
        for (int i = 0; stack && i < L; i++)
            free(stack[i]);
        free(stack);
        free(local);
    }
    return fail ? -1 : 0;
}

/* State (logical, including Pauli noise and global phases) of node m at
 * `level` after its subcircuit, computed along its ancestor chain. */
int orc_node_state_k(int n, int G, const int *kind, const int *q0, const int *q1,
                     const double *theta, const double *mat, double p1, double p2, const double *kr,
                     uint64_t seed, int L, const uint64_t *arity, const int *split, int level,
                     uint64_t m, double *psi_out);

int orc_node_state(int n, int G, const int *kind, const int *q0, const int *q1,
                   const double *theta, const double *mat, double p1, double p2, uint64_t seed,
                   int L, const uint64_t *arity, const int *split, int level, uint64_t m,
                   double *psi_out)
{
    return orc_node_state_k(n, G, kind, q0, q1, theta, mat, p1, p2, NULL, seed, L, arity, split, level, m,
                            psi_out);
}

/* As orc_node_state, with the non-unitary channels of `kr` (NULL = none). */
int orc_node_state_k(int n, int G, const int *kind, const int *q0, const int *q1,
                     const double *theta, const double *mat, double p1, double p2, const double *kr,
                     uint64_t seed, int L, const uint64_t *arity, const int *split, int level,
                     uint64_t m, double *psi_out)
{
    circuit c = {n, G, kind, q0, q1, theta, mat};
    (void)L;
    uint64_t chain[64];
    chain[level] = m;
    for (int i = level; i > 0; i--)
        chain[i - 1] = chain[i] / arity[i];
    uint64_t dim = (uint64_t)1 << n;
    cplx *psi = calloc(dim, sizeof(cplx));
    if (!psi)
        return -1;
    psi[0] = 1.0;
    for (int i = 0; i <= level; i++)
        for (int g = split[i]; g < split[i + 1]; g++) {
            apply_gate(psi, &c, g);
            apply_noise(psi, &c, g, seed, chain[i], p1, p2);
            apply_kraus(psi, &c, g, seed, chain[i], kr);
        }
    memcpy(psi_out, psi, dim * sizeof(cplx));
    free(psi);
    return 0;
}

/* Outcome (after readout error) of a single leaf, computed along its chain.
 * Lets tests check arbitrary leaves of trees too large to run in full. */
int64_t orc_leaf_outcome_k(int n, int G, const int *kind, const int *q0, const int *q1,
                           const double *theta, const double *mat, double p1, double p2, double pm,
                           const double *kr, uint64_t seed, int L, const uint64_t *arity,
                           const int *split, uint64_t leaf);

int64_t orc_leaf_outcome(int n, int G, const int *kind, const int *q0, const int *q1,
                         const double *theta, const double *mat, double p1, double p2, double pm,
                         uint64_t seed, int L, const uint64_t *arity, const int *split,
                         uint64_t leaf)
{
    return orc_leaf_outcome_k(n, G, kind, q0, q1, theta, mat, p1, p2, pm, NULL, seed, L, arity, split, leaf);
}

/* As orc_leaf_outcome, with the non-unitary channels of `kr` (NULL = none). */
int64_t orc_leaf_outcome_k(int n, int G, const int *kind, const int *q0, const int *q1,
                           const double *theta, const double *mat, double p1, double p2, double pm,
                           const double *kr, uint64_t seed, int L, const uint64_t *arity,
                           const int *split, uint64_t leaf)
{
    uint64_t dim = (uint64_t)1 << n;
    double *psi = malloc(2 * dim * sizeof(double));
    if (!psi)
        return -1;
    orc_node_state_k(n, G, kind, q0, q1, theta, mat, p1, p2, kr, seed, L, arity, split, L - 1, leaf,
                     psi);
    uint64_t y = sample_index((const cplx *)psi, n, orc_measure_u(seed, leaf));
    y ^= orc_readout_mask(seed, leaf, n, pm);
    free(psi);
    return (int64_t)y;
}

/* Noise assignment of node m at `level`: out[g - split[level]] = Pauli index or 0. */
void orc_node_noise(int G, const int *kind, double p1, double p2, uint64_t seed,
                    const int *split, int level, uint64_t m, int *out)
{
    (void)G;
    for (int g = split[level]; g < split[level + 1]; g++) {
        int two = gate_arity(kind[g]) == 2;
        out[g - split[level]] = orc_noise_draw(seed, m, (uint32_t)g, two ? p2 : p1, two ? 15 : 3);
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
