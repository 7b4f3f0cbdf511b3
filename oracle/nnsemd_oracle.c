/*
 * TEST INFRASTRUCTURE -- the CPU oracle of NNS-EMD.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load this file's
 * library; the product path never does.
 *
 * A plain, deliberately slow statement of NNS-EMD with the greedy protocol
 * (Alg. 1, Sec. III-A), written from the method's description.  Each round
 * looks only at the points that still hold weight.  Every such consumer
 * picks its nearest such supplier (the NNS operation), by a full double loop.
 * Every supplier then takes the consumers that picked it, orders them by
 * distance (greedy protocol) or by a seeded random key (random protocol),
 * and hands each in turn the smaller of the two residuals until its own
 * residual is gone, adding that amount times the ground distance to R and
 * to the plan entry.  Rounds repeat until one side has no weight left.
 *
 * Readings of the paper taken here (the paper is silent or garbled on them):
 *  - Inner greedy loop: every consumer of the sorted group is visited while
 *    s_i > 0 (the printed loop bound "l < |a_i|" would skip the last one; the
 *    prose of Sec. III-A serves the group until s_i is spent).
 *  - Ties in the argmin go to the lowest supplier index; ties in the greedy
 *    order go to the lowest consumer index.
 *  - The loop stops when either active set is empty: in floating point the
 *    two residual totals need not reach zero together.  A point retires when
 *    its residual is exactly 0; since f = min(s, c), the smaller side always
 *    reaches exactly 0, so every round retires at least one point.
 *  - The argmin and the greedy order use the squared Euclidean distance for
 *    the L2 and squared-L2 metrics (same order), the L1 sum for L1.  The cost
 *    D_ij uses the requested metric (sqrt for L2) in FP64.
 *  - Decision precision: the paper fixes none.  decide_fp32 = 0 takes every
 *    decision in FP64.  decide_fp32 = 1 takes the argmin and the greedy order
 *    in FP32 with one fixed operation order (below), the precision of the
 *    single-precision GPU kernels, and checks each such decision against the
 *    FP64 one: where the two pick differently, the FP64 distances must be
 *    within 1e-6 relative (a near-tie) or the call reports a violation.
 *
 *  - Random protocol (Sec. III-A names it; the paper fixes no generator):
 *    a group is served in ascending order of a 32-bit key per consumer, the
 *    upper half of SplitMix64 output number c + 1 of the generator seeded
 *    with `seed`, for the counter c = (t << 32) | j (round t from 0, original
 *    consumer index j); equal keys go to the lower j.
 *
 * FP32 squared distance:  t_k = fl32(x_k - y_k);  acc = fl32(t_0 * t_0);
 *                         acc = fmaf(t_k, t_k, acc) for k = 1..d-1.
 * FP32 L1 distance:       acc = |t_0|; acc = fl32(acc + |t_k|).
 * FP64 forms: the same steps in double (fma for the squared form).
 *
 * Mass bookkeeping is FP64.  Weights arrive already normalised (the Python
 * wrapper divides by the correctly rounded total).  Build with
 * -ffp-contract=off so that no multiply-add is fused behind our back.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { METRIC_L2 = 0, METRIC_SQL2 = 1, METRIC_L1 = 2 };

enum {
    ORC_OK = 0,
    ORC_ERR_ARG = 1,
    ORC_ERR_ALLOC = 5,
    ORC_ERR_ITER = 7,
    ORC_ERR_CAPACITY = 9
};

#define NEAR_TIE_REL 1e-6

static float key32(const float *xi, const float *yj, int d, int metric)
{
    if (metric == METRIC_L1) {
        float acc = fabsf(xi[0] - yj[0]);
        for (int k = 1; k < d; ++k)
            acc = acc + fabsf(xi[k] - yj[k]);
        return acc;
    }
    float t = xi[0] - yj[0];
    float acc = t * t;
    for (int k = 1; k < d; ++k) {
        float u = xi[k] - yj[k];
        acc = fmaf(u, u, acc);
    }
    return acc;
}

static double key64(const float *xi, const float *yj, int d, int metric)
{
    if (metric == METRIC_L1) {
        double acc = fabs((double)xi[0] - (double)yj[0]);
        for (int k = 1; k < d; ++k)
            acc = acc + fabs((double)xi[k] - (double)yj[k]);
        return acc;
    }
    double t = (double)xi[0] - (double)yj[0];
    double acc = t * t;
    for (int k = 1; k < d; ++k) {
        double u = (double)xi[k] - (double)yj[k];
        acc = fma(u, u, acc);
    }
    return acc;
}

/* Ground distance D_ij of the cost (Eq. objective), FP64. */
static double cost_dist(const float *xi, const float *yj, int d, int metric)
{
    double k = key64(xi, yj, d, metric);
    return metric == METRIC_L2 ? sqrt(k) : k;
}

/* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the generator adds 0x9E3779B97F4A7C15 to its
 * state per step and outputs the state passed through the mixing function
 * below, so output number k (k >= 1) of the generator seeded with `seed` is
 * mix(seed + k * 0x9E3779B97F4A7C15), all arithmetic modulo 2^64. */
uint64_t oracle_splitmix64_output(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Random-protocol key of consumer j in round t (see the header). */
static uint32_t rp_key(uint64_t seed, int64_t t, int64_t j)
{
    const uint64_t c = ((uint64_t)t << 32) | (uint64_t)(uint32_t)j;
    return (uint32_t)(oracle_splitmix64_output(seed, c + 1) >> 32);
}

/* One member of a supplier's group a_i: its consumer and its sort keys. */
typedef struct {
    int64_t j;
    float k32;
    double k64;
    int use32;
    int random;     /* random protocol: order by rk */
    uint32_t rk;
} member_t;

static int cmp_member(const void *pa, const void *pb)
{
    const member_t *a = (const member_t *)pa, *b = (const member_t *)pb;
    if (a->random) {
        if (a->rk < b->rk) return -1;
        if (a->rk > b->rk) return 1;
    } else if (a->use32) {
        if (a->k32 < b->k32) return -1;
        if (a->k32 > b->k32) return 1;
    } else {
        if (a->k64 < b->k64) return -1;
        if (a->k64 > b->k64) return 1;
    }
    return (a->j > b->j) - (a->j < b->j);
}

typedef struct {
    int64_t rounds;
    int64_t pair_evals;      /* sum over rounds of m_t * n_t */
    int64_t nnz;
    int64_t near_ties;       /* FP32 decisions that differ from FP64 ones */
    int64_t violations;      /* ... by more than the near-tie allowance */
    double max_rel_gap;      /* largest relative FP64 gap among those */
    double cost_seq;         /* R accumulated in Alg. 1's order */
    double leftover_s;       /* sum of supplier residuals left at the end */
    double leftover_c;       /* sum of consumer residuals left at the end */
} oracle_stats;

/*
 * x [m*d], y [n*d] float32 row-major; s [m], c [n] normalised FP64 weights
 * (modified in place: they end as the residuals).
 * Plan outputs (capacity plan_cap): pi, pj, pf, pterm (= f * D_ij).
 * Optional per-round outputs (capacity round_cap, may be NULL): m_t, n_t.
 * Optional NN trace (capacity trace_cap, may be NULL): for each round and
 * each active consumer in ascending j, (j, NNS(j)) appended.
 */
int oracle_nnsemd(int64_t m, int64_t n, int32_t d, const float *x, double *s,
                  const float *y, double *c, int32_t metric, int32_t decide_fp32,
                  int32_t protocol, uint64_t seed,
                  int64_t plan_cap, int32_t *pi, int32_t *pj, double *pf, double *pterm,
                  int64_t round_cap, int64_t *m_t, int64_t *n_t,
                  int64_t trace_cap, int32_t *trace_j, int32_t *trace_nn,
                  oracle_stats *st)
{
    if (m < 0 || n < 0 || d < 1 || !st || (metric < 0 || metric > 2) || protocol < 0 || protocol > 1)
        return ORC_ERR_ARG;
    memset(st, 0, sizeof(*st));
    int64_t *I = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t *J = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *nn = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    member_t *grp = (member_t *)malloc(sizeof(member_t) * (size_t)(n > 0 ? n : 1));
    if (!I || !J || !nn || !grp) {
        free(I); free(J); free(nn); free(grp);
        return ORC_ERR_ALLOC;
    }
    int rc = ORC_OK;
    int64_t trace_len = 0;
    const int64_t round_limit = m + n;

    for (;;) {
        /* active index sets, ascending */
        int64_t mt = 0, nt = 0;
        for (int64_t i = 0; i < m; ++i)
            if (s[i] > 0.0) I[mt++] = i;
        for (int64_t j = 0; j < n; ++j)
            if (c[j] > 0.0) J[nt++] = j;
        if (mt == 0 || nt == 0)
            break;
        if (st->rounds >= round_limit) { rc = ORC_ERR_ITER; break; }
        if (m_t && st->rounds < round_cap) { m_t[st->rounds] = mt; n_t[st->rounds] = nt; }
        st->pair_evals += mt * nt;

        /* NNS operation: nearest active supplier of every active consumer */
        for (int64_t q = 0; q < nt; ++q) {
            const int64_t j = J[q];
            const float *yj = y + j * d;
            int64_t best64_i = -1, best32_i = -1;
            double best64 = 0.0;
            float best32 = 0.0f;
            for (int64_t p = 0; p < mt; ++p) {
                const int64_t i = I[p];
                const float *xi = x + i * d;
                double k = key64(xi, yj, d, metric);
                if (best64_i < 0 || k < best64) { best64 = k; best64_i = i; }
                if (decide_fp32) {
                    float k2 = key32(xi, yj, d, metric);
                    if (best32_i < 0 || k2 < best32) { best32 = k2; best32_i = i; }
                }
            }
            int64_t pick = best64_i;
            if (decide_fp32) {
                pick = best32_i;
                if (best32_i != best64_i) {
                    double k = key64(x + best32_i * d, yj, d, metric);
                    double gap = (k - best64) / fmax(best64, 1e-30);
                    st->near_ties++;
                    if (gap > st->max_rel_gap) st->max_rel_gap = gap;
                    if (gap > NEAR_TIE_REL) st->violations++;
                }
            }
            nn[q] = pick;
            if (trace_j && trace_len < trace_cap) {
                trace_j[trace_len] = (int32_t)j;
                trace_nn[trace_len] = (int32_t)pick;
            }
            trace_len++;
        }

        /* flow & cost, greedy protocol, one supplier at a time */
        for (int64_t p = 0; p < mt; ++p) {
            const int64_t i = I[p];
            const float *xi = x + i * d;
            int64_t L = 0;
            for (int64_t q = 0; q < nt; ++q) {
                if (nn[q] != i) continue;
                member_t e;
                e.j = J[q];
                e.k64 = key64(xi, y + e.j * d, d, metric);
                e.k32 = decide_fp32 ? key32(xi, y + e.j * d, d, metric) : 0.0f;
                e.use32 = decide_fp32;
                e.random = protocol == 1;
                e.rk = protocol == 1 ? rp_key(seed, st->rounds, e.j) : 0u;
                grp[L++] = e;
            }
            if (L == 0) continue;
            qsort(grp, (size_t)L, sizeof(member_t), cmp_member);
            if (decide_fp32 && protocol == 0) {
                /* every inversion against the FP64 order must be a near-tie */
                double run_max = grp[0].k64;
                for (int64_t l = 1; l < L; ++l) {
                    if (run_max > grp[l].k64) {
                        double gap = (run_max - grp[l].k64) / fmax(grp[l].k64, 1e-30);
                        st->near_ties++;
                        if (gap > st->max_rel_gap) st->max_rel_gap = gap;
                        if (gap > NEAR_TIE_REL) st->violations++;
                    }
                    if (grp[l].k64 > run_max) run_max = grp[l].k64;
                }
            }
            for (int64_t l = 0; l < L && s[i] > 0.0; ++l) {
                const int64_t j = grp[l].j;
                double f = s[i] < c[j] ? s[i] : c[j];
                s[i] = s[i] - f;
                c[j] = c[j] - f;
                double D = cost_dist(xi, y + j * d, d, metric);
                double term = f * D;
                st->cost_seq = st->cost_seq + term;
                if (st->nnz >= plan_cap) { rc = ORC_ERR_CAPACITY; goto done; }
                pi[st->nnz] = (int32_t)i;
                pj[st->nnz] = (int32_t)j;
                pf[st->nnz] = f;
                pterm[st->nnz] = term;
                st->nnz++;
            }
        }
        st->rounds++;
    }
done:
    for (int64_t i = 0; i < m; ++i) st->leftover_s += s[i];
    for (int64_t j = 0; j < n; ++j) st->leftover_c += c[j];
    free(I); free(J); free(nn); free(grp);
    return rc;
}

/* Number of trace entries the last shape needs is not known in advance; the
 * wrapper grows its buffers and retries.  This helper reports the struct size
 * so the wrapper can check its ctypes layout. */
int oracle_stats_size(void) { return (int)sizeof(oracle_stats); }

/*
 * Nearest of k points (centroids) for each of N points: the FP32 squared
 * distance key of the NNS operation (key32, metric squared L2), lowest
 * centroid index on ties.  The assignment step of the k-means colour
 * quantisation that precedes the colour-transfer EMD (Sec. IV-D).
 */
void oracle_assign(const float *pts, int64_t N, const float *cent, int64_t k, int32_t d, int32_t *out)
{
    for (int64_t p = 0; p < N; ++p) {
        float best = 0.0f;
        int64_t bi = -1;
        for (int64_t c = 0; c < k; ++c) {
            const float v = key32(cent + c * d, pts + p * d, d, METRIC_SQL2);
            if (bi < 0 || v < best) { best = v; bi = c; }
        }
        out[p] = (int32_t)bi;
    }
}
