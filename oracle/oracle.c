/*
 * CPU oracle for the GAS superstep engine. TEST INFRASTRUCTURE ONLY: the
 * tests, the smoke check and the benchmark's CPU-baseline leg call it; the
 * product path never does.
 *
 * Plain, single-threaded, unblocked C99. It shares no code with the CUDA path.
 * Every routine works straight on the COO edge list as given (no sorting, no
 * CSC, no tiling): one BSP superstep (Section IV-A1: MSGGen, MSGMerge,
 * MSGApply, in the BSP order Gen -> Merge -> Apply of Section IV-B2) reads
 * only the previous superstep's vertex values (Jacobi).
 *
 * The paper names the algorithms (Section V-A: SSSP Bellman-Ford, PageRank,
 * Label Propagation) but gives no formulas; the definitions below are the
 * textbook ones, with these readings:
 *   SSSP  d_0[s]=0, else INF=0xFFFFFFFF; per superstep, over all edges (u,v,w)
 *         with d[u] != INF: m[v] = min(m[v], d[u]+w) in 64-bit; then
 *         d'[v] = min(d[v], m[v]). Stop after the first superstep that
 *         changes nothing.
 *   CC    (label propagation read as min-label propagation) l_0[v]=v;
 *         m[v] = min over in-edges of l[u]; l'[v] = min(l[v], m[v]); stop as
 *         for SSSP.
 *   PR    N=|V|, r_0=1/N, D_t = sum of r_t over out-degree-0 vertices,
 *         r_{t+1}[v] = (1-d)/N + d*(sum_{(u,v)} r_t[u]/outdeg(u) + D_t/N),
 *         fixed number of supersteps, fp64.
 *   PPR   r_0 = e_s, r_{t+1} = (1-d) e_s + d*(A^T D^-1 r_t + D_t e_s), fp64.
 *   LP    (label propagation read as synchronous mode-label propagation, the
 *         paper's LP workload, capped at 15 supersteps in Section V-A)
 *         l_0[v]=v; v's new label is the label carried by the most in-edges
 *         (u,v) (message l[u]), ties to the smallest label; a vertex without
 *         in-edges keeps its label. Stop after a superstep that changes
 *         nothing, or after max_steps.
 * Multi-edges count in out-degrees and in merges; self-loops are kept.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_INF 0xFFFFFFFFu

/* ---------------------------------------------------------------- SSSP ---- */

/* One Jacobi Bellman-Ford superstep: d_out from d_in. Returns #changed. */
uint64_t orc_sssp_step(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                       const uint32_t* w, const uint32_t* d_in, uint32_t* d_out,
                       uint64_t* msg /* scratch, n entries */) {
    for (uint64_t v = 0; v < n; ++v) msg[v] = UINT64_MAX;        /* MSGMerge identity */
    for (uint64_t e = 0; e < m; ++e) {                             /* MSGGen + MSGMerge */
        const uint32_t u = src[e];
        if (d_in[u] == ORC_INF) continue;
        const uint64_t cand = (uint64_t)d_in[u] + (uint64_t)w[e];
        if (cand < msg[dst[e]]) msg[dst[e]] = cand;
    }
    uint64_t changed = 0;
    for (uint64_t v = 0; v < n; ++v) {                             /* MSGApply */
        uint64_t nv = d_in[v];
        if (msg[v] < nv) nv = msg[v];
        if (nv >= (uint64_t)ORC_INF) nv = ORC_INF; /* unreachable with the workloads' bounds */
        d_out[v] = (uint32_t)nv;
        changed += (d_out[v] != d_in[v]);
    }
    return changed;
}

/*
 * Full run from `source` until a superstep changes nothing (or max_steps).
 * Returns supersteps executed (including the final no-change one), or -1 on
 * allocation failure / overflow of a distance into INF.
 * changed_per_step (nullable, max_steps entries) receives each step's count.
 */
int64_t orc_sssp(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                 const uint32_t* w, uint32_t source, uint32_t max_steps,
                 uint32_t* dist, uint64_t* changed_per_step) {
    uint32_t* other = (uint32_t*)malloc(n * sizeof(uint32_t) + 4);
    uint64_t* msg = (uint64_t*)malloc(n * sizeof(uint64_t) + 8);
    if (!other || !msg) { free(other); free(msg); return -1; }
    for (uint64_t v = 0; v < n; ++v) dist[v] = ORC_INF;
    if (source < n) dist[source] = 0;
    uint32_t* cur = dist; uint32_t* nxt = other;
    int64_t steps = 0;
    for (uint32_t t = 0; t < max_steps; ++t) {
        const uint64_t c = orc_sssp_step(n, m, src, dst, w, cur, nxt, msg);
        if (changed_per_step) changed_per_step[t] = c;
        ++steps;
        uint32_t* tmp = cur; cur = nxt; nxt = tmp;
        if (c == 0) break;
    }
    if (cur != dist) memcpy(dist, cur, n * sizeof(uint32_t));
    free(other); free(msg);
    return steps;
}

/* ------------------------------------------------------------------ CC ---- */

uint64_t orc_cc_step(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                     const uint32_t* l_in, uint32_t* l_out, uint32_t* msg /* scratch, n */) {
    for (uint64_t v = 0; v < n; ++v) msg[v] = ORC_INF;            /* MSGMerge identity */
    for (uint64_t e = 0; e < m; ++e) {                             /* MSGGen + MSGMerge(min) */
        const uint32_t x = l_in[src[e]];
        if (x < msg[dst[e]]) msg[dst[e]] = x;
    }
    uint64_t changed = 0;
    for (uint64_t v = 0; v < n; ++v) {                             /* MSGApply(min) */
        l_out[v] = msg[v] < l_in[v] ? msg[v] : l_in[v];
        changed += (l_out[v] != l_in[v]);
    }
    return changed;
}

int64_t orc_cc(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
               uint32_t max_steps, uint32_t* labels, uint64_t* changed_per_step) {
    uint32_t* other = (uint32_t*)malloc(n * sizeof(uint32_t) + 4);
    uint32_t* msg = (uint32_t*)malloc(n * sizeof(uint32_t) + 4);
    if (!other || !msg) { free(other); free(msg); return -1; }
    for (uint64_t v = 0; v < n; ++v) labels[v] = (uint32_t)v;
    uint32_t* cur = labels; uint32_t* nxt = other;
    int64_t steps = 0;
    for (uint32_t t = 0; t < max_steps; ++t) {
        const uint64_t c = orc_cc_step(n, m, src, dst, cur, nxt, msg);
        if (changed_per_step) changed_per_step[t] = c;
        ++steps;
        uint32_t* tmp = cur; cur = nxt; nxt = tmp;
        if (c == 0) break;
    }
    if (cur != labels) memcpy(labels, cur, n * sizeof(uint32_t));
    free(other); free(msg);
    return steps;
}

/* ------------------------------------------------------------------ LP ---- */

static int orc_cmp_u64(const void* a, const void* b) {
    const uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/*
 * One synchronous mode-label superstep: l_out from l_in. MSGGen sends l_in[u]
 * along every edge (u,v); MSGMerge takes the mode of v's messages (the
 * (v, label) pairs are sorted, so equal labels of v are adjacent and labels
 * ascend: the first run of the largest length is the smallest label among
 * the most frequent); MSGApply sets it, or keeps l_in[v] without messages.
 * Returns #changed.
 */
uint64_t orc_lp_step(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                     const uint32_t* l_in, uint32_t* l_out, uint64_t* pairs /* scratch, m entries */) {
    for (uint64_t e = 0; e < m; ++e)                               /* MSGGen */
        pairs[e] = ((uint64_t)dst[e] << 32) | (uint64_t)l_in[src[e]];
    qsort(pairs, (size_t)m, sizeof(uint64_t), orc_cmp_u64);
    for (uint64_t v = 0; v < n; ++v) l_out[v] = l_in[v];          /* no messages: keep */
    uint64_t i = 0;
    while (i < m) {                                                /* MSGMerge(mode) + MSGApply */
        const uint64_t v = pairs[i] >> 32;
        uint64_t best_count = 0;
        uint32_t best_label = 0;
        while (i < m && (pairs[i] >> 32) == v) {
            uint64_t k = i;
            while (k < m && pairs[k] == pairs[i]) ++k;
            if (k - i > best_count) {                              /* strict: ties keep the smaller label */
                best_count = k - i;
                best_label = (uint32_t)pairs[i];
            }
            i = k;
        }
        l_out[v] = best_label;
    }
    uint64_t changed = 0;
    for (uint64_t v = 0; v < n; ++v) changed += (l_out[v] != l_in[v]);
    return changed;
}

int64_t orc_lp(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
               uint32_t max_steps, uint32_t* labels, uint64_t* changed_per_step) {
    uint32_t* other = (uint32_t*)malloc(n * sizeof(uint32_t) + 4);
    uint64_t* pairs = (uint64_t*)malloc(m * sizeof(uint64_t) + 8);
    if (!other || !pairs) { free(other); free(pairs); return -1; }
    for (uint64_t v = 0; v < n; ++v) labels[v] = (uint32_t)v;
    uint32_t* cur = labels; uint32_t* nxt = other;
    int64_t steps = 0;
    for (uint32_t t = 0; t < max_steps; ++t) {
        const uint64_t c = orc_lp_step(n, m, src, dst, cur, nxt, pairs);
        if (changed_per_step) changed_per_step[t] = c;
        ++steps;
        uint32_t* tmp = cur; cur = nxt; nxt = tmp;
        if (c == 0) break;
    }
    if (cur != labels) memcpy(labels, cur, n * sizeof(uint32_t));
    free(other); free(pairs);
    return steps;
}

/* ----------------------------------------------------------- PageRank ---- */

void orc_outdeg(uint64_t n, uint64_t m, const uint32_t* src, uint64_t* outdeg) {
    for (uint64_t v = 0; v < n; ++v) outdeg[v] = 0;
    for (uint64_t e = 0; e < m; ++e) outdeg[src[e]] += 1;
}

/*
 * One PageRank superstep in fp64: r_out from r_in. Returns the dangling mass
 * D_t of r_in; *l1 receives sum |r_out - r_in|.
 */
double orc_pr_step(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                   const uint64_t* outdeg, double damping, const double* r_in,
                   double* r_out, double* l1) {
    double dangling = 0.0;
    for (uint64_t v = 0; v < n; ++v)
        if (outdeg[v] == 0) dangling += r_in[v];
    for (uint64_t v = 0; v < n; ++v) r_out[v] = 0.0;               /* Merge(sum) identity */
    for (uint64_t e = 0; e < m; ++e)                               /* Gen + Merge */
        r_out[dst[e]] += r_in[src[e]] / (double)outdeg[src[e]];
    const double N = (double)n;
    double s = 0.0;
    for (uint64_t v = 0; v < n; ++v) {                             /* Apply */
        r_out[v] = (1.0 - damping) / N + damping * (r_out[v] + dangling / N);
        s += fabs(r_out[v] - r_in[v]);
    }
    if (l1) *l1 = s;
    return dangling;
}

/*
 * `iters` supersteps from r_0 = 1/N. rank receives r_iters. l1_per_step and
 * dangling_per_step (nullable, iters entries) receive sum|r_{t+1}-r_t| and
 * D_t. Returns 0, or -1 on allocation failure.
 */
int orc_pagerank(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                 double damping, uint32_t iters, double* rank,
                 double* l1_per_step, double* dangling_per_step) {
    uint64_t* outdeg = (uint64_t*)malloc(n * sizeof(uint64_t) + 8);
    double* other = (double*)malloc(n * sizeof(double) + 8);
    if (!outdeg || !other) { free(outdeg); free(other); return -1; }
    orc_outdeg(n, m, src, outdeg);
    for (uint64_t v = 0; v < n; ++v) rank[v] = 1.0 / (double)n;
    double* cur = rank; double* nxt = other;
    for (uint32_t t = 0; t < iters; ++t) {
        double l1 = 0.0;
        const double dang = orc_pr_step(n, m, src, dst, outdeg, damping, cur, nxt, &l1);
        if (l1_per_step) l1_per_step[t] = l1;
        if (dangling_per_step) dangling_per_step[t] = dang;
        double* tmp = cur; cur = nxt; nxt = tmp;
    }
    if (cur != rank) memcpy(rank, cur, n * sizeof(double));
    free(outdeg); free(other);
    return 0;
}

/*
 * Personalized PageRank from `source`: teleport and dangling mass both return
 * to the source. `iters` supersteps from r_0 = e_s, fp64.
 */
int orc_ppr(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
            uint32_t source, double damping, uint32_t iters, double* rank) {
    uint64_t* outdeg = (uint64_t*)malloc(n * sizeof(uint64_t) + 8);
    double* other = (double*)malloc(n * sizeof(double) + 8);
    if (!outdeg || !other || source >= n) { free(outdeg); free(other); return -1; }
    orc_outdeg(n, m, src, outdeg);
    for (uint64_t v = 0; v < n; ++v) rank[v] = 0.0;
    rank[source] = 1.0;
    double* cur = rank; double* nxt = other;
    for (uint32_t t = 0; t < iters; ++t) {
        double dangling = 0.0;
        for (uint64_t v = 0; v < n; ++v)
            if (outdeg[v] == 0) dangling += cur[v];
        for (uint64_t v = 0; v < n; ++v) nxt[v] = 0.0;
        for (uint64_t e = 0; e < m; ++e)
            nxt[dst[e]] += cur[src[e]] / (double)outdeg[src[e]];
        for (uint64_t v = 0; v < n; ++v) nxt[v] = damping * nxt[v];
        nxt[source] += (1.0 - damping) + damping * dangling;
        double* tmp = cur; cur = nxt; nxt = tmp;
    }
    if (cur != rank) memcpy(rank, cur, n * sizeof(double));
    free(outdeg); free(other);
    return 0;
}
