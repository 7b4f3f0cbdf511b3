/*
 * TEST INFRASTRUCTURE -- the multi-core twin of the CPU oracle (see
 * nnsemd_oracle.c, which this file includes so that both use the very same
 * distance, cost, generator and ordering helpers).  Only the tests and the
 * benchmark's CPU-baseline leg load the library built from this file.
 */
#include "nnsemd_oracle.c"

/*
 * The multi-core twin of oracle_nnsemd (used to time the oracle on all host
 * cores and to check large parity cases in reasonable time).  It computes
 * the same thing with the same helpers and the same operations, reorganised
 * only where the order cannot change a result:
 *  - the NNS operation runs over the consumers in parallel (each consumer's
 *    scan is the serial one; the near-tie counts are sums and a maximum);
 *  - the groups a_i are built by one counting pass over the consumers in
 *    ascending order instead of one scan of all consumers per supplier, and
 *    each group is sorted in parallel (the sort order is total: ties go to
 *    the lower consumer index, so any sort gives the same sequence);
 *  - the flows run serially in ascending supplier order, exactly as in
 *    oracle_nnsemd, so residuals, plan entries and cost_seq are the same.
 * threads <= 0 uses every core OpenMP reports.  Built without OpenMP, the
 * pragmas are ignored and the twin runs on one core.
 */
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_omp_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oracle_nnsemd_omp(int64_t m, int64_t n, int32_t d, const float *x, double *s,
                      const float *y, double *c, int32_t metric, int32_t decide_fp32,
                      int32_t protocol, uint64_t seed,
                      int64_t plan_cap, int32_t *pi, int32_t *pj, double *pf, double *pterm,
                      int64_t round_cap, int64_t *m_t, int64_t *n_t,
                      int64_t trace_cap, int32_t *trace_j, int32_t *trace_nn,
                      int32_t threads, oracle_stats *st)
{
    if (m < 0 || n < 0 || d < 1 || !st || (metric < 0 || metric > 2) || protocol < 0 || protocol > 1)
        return ORC_ERR_ARG;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    memset(st, 0, sizeof(*st));
    const size_t mm = (size_t)(m > 0 ? m : 1), nn1 = (size_t)(n > 0 ? n : 1);
    int64_t *I = (int64_t *)malloc(sizeof(int64_t) * mm);
    int64_t *J = (int64_t *)malloc(sizeof(int64_t) * nn1);
    int64_t *nn = (int64_t *)malloc(sizeof(int64_t) * nn1);
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * mm);       /* supplier index -> active position */
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (mm + 1)); /* group offsets by position */
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * mm);
    member_t *grp = (member_t *)malloc(sizeof(member_t) * nn1);
    if (!I || !J || !nn || !pos || !off || !fill || !grp) {
        free(I); free(J); free(nn); free(pos); free(off); free(fill); free(grp);
        return ORC_ERR_ALLOC;
    }
    int rc = ORC_OK;
    int64_t trace_len = 0;
    const int64_t round_limit = m + n;

    for (;;) {
        int64_t mt = 0, nt = 0;
        for (int64_t i = 0; i < m; ++i)
            if (s[i] > 0.0) { pos[i] = mt; I[mt++] = i; }
        for (int64_t j = 0; j < n; ++j)
            if (c[j] > 0.0) J[nt++] = j;
        if (mt == 0 || nt == 0)
            break;
        if (st->rounds >= round_limit) { rc = ORC_ERR_ITER; break; }
        if (m_t && st->rounds < round_cap) { m_t[st->rounds] = mt; n_t[st->rounds] = nt; }
        st->pair_evals += mt * nt;

        /* NNS operation, one consumer per iteration */
        int64_t ties = 0, viol = 0;
        double gapmax = st->max_rel_gap;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : ties, viol) reduction(max : gapmax)
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
                    ties++;
                    if (gap > gapmax) gapmax = gap;
                    if (gap > NEAR_TIE_REL) viol++;
                }
            }
            nn[q] = pick;
        }
        for (int64_t q = 0; q < nt; ++q) {
            if (trace_j && trace_len < trace_cap) {
                trace_j[trace_len] = (int32_t)J[q];
                trace_nn[trace_len] = (int32_t)nn[q];
            }
            trace_len++;
        }

        /* groups a_i: counting pass in ascending consumer order */
        for (int64_t p = 0; p <= mt; ++p) off[p] = 0;
        for (int64_t q = 0; q < nt; ++q) off[pos[nn[q]] + 1]++;
        for (int64_t p = 0; p < mt; ++p) { off[p + 1] += off[p]; fill[p] = off[p]; }
        for (int64_t q = 0; q < nt; ++q) {
            const int64_t p = pos[nn[q]];
            grp[fill[p]++].j = J[q];
        }
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : ties, viol) reduction(max : gapmax)
        for (int64_t p = 0; p < mt; ++p) {
            const int64_t L = off[p + 1] - off[p];
            if (L == 0) continue;
            member_t *g = grp + off[p];
            const float *xi = x + I[p] * d;
            for (int64_t l = 0; l < L; ++l) {
                member_t *e = g + l;
                e->k64 = key64(xi, y + e->j * d, d, metric);
                e->k32 = decide_fp32 ? key32(xi, y + e->j * d, d, metric) : 0.0f;
                e->use32 = decide_fp32;
                e->random = protocol == 1;
                e->rk = protocol == 1 ? rp_key(seed, st->rounds, e->j) : 0u;
            }
            qsort(g, (size_t)L, sizeof(member_t), cmp_member);
            if (decide_fp32 && protocol == 0) {
                double run_max = g[0].k64;
                for (int64_t l = 1; l < L; ++l) {
                    if (run_max > g[l].k64) {
                        double gap = (run_max - g[l].k64) / fmax(g[l].k64, 1e-30);
                        ties++;
                        if (gap > gapmax) gapmax = gap;
                        if (gap > NEAR_TIE_REL) viol++;
                    }
                    if (g[l].k64 > run_max) run_max = g[l].k64;
                }
            }
        }
        st->near_ties += ties;
        st->violations += viol;
        st->max_rel_gap = gapmax;

        /* flows, serially in ascending supplier order */
        for (int64_t p = 0; p < mt; ++p) {
            const int64_t i = I[p];
            const float *xi = x + i * d;
            const member_t *g = grp + off[p];
            const int64_t L = off[p + 1] - off[p];
            for (int64_t l = 0; l < L && s[i] > 0.0; ++l) {
                const int64_t j = g[l].j;
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
    free(I); free(J); free(nn); free(pos); free(off); free(fill); free(grp);
    return rc;
}

