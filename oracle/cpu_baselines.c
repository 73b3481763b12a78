/*
 * CPU baselines timed by bench.py beside the GPU numbers. NOT the oracle:
 * nothing here is used to check a result of the CUDA path, and parity never
 * depends on it (the oracle, oracle.c, stays plain single-threaded C).
 *
 *  - cb_pagerank_pull: PageRank (the same recurrence as the oracle: r_0 = 1/N,
 *    dangling mass spread evenly, fp64) pulled by destination over a CSC on
 *    all host cores with OpenMP; each thread owns whole destinations, so no
 *    atomics are needed.
 *  - cb_minlabel_pull: the min-merge supersteps (SSSP relaxation or CC
 *    labels) pulled by destination over a CSC on all cores, Jacobi, until a
 *    superstep changes nothing.
 *  - cb_dijkstra: textbook Dijkstra with a binary heap over a CSR (one core),
 *    the classic sequential algorithm the SSSP supersteps are compared with.
 *  - cb_union_find: connected components by union-find with path halving
 *    and union by smaller root id (one core): every vertex ends labelled with
 *    the smallest id of its component, as min-label propagation gives.
 *
 * Compiled with -fopenmp into its own library; the caller chooses the thread
 * count (omp_set_num_threads) and reports it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int cb_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void cb_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* iters supersteps from r = 1/N; col_ptr[n+1] (u64) and src[] are the CSC of
 * in-edges, outdeg[u] the out-degree; r_out[n] receives the ranks. Returns 0,
 * or -1 when scratch cannot be allocated. */
int cb_pagerank_pull(uint64_t n, const uint64_t* col_ptr, const uint32_t* src, const uint32_t* outdeg,
                     double damping, uint32_t iters, double* r_out) {
    double* r = r_out;
    double* c = (double*)malloc(sizeof(double) * (n ? n : 1));
    if (!c) return -1;
    const double inv_n = 1.0 / (double)n;
    for (uint64_t v = 0; v < n; ++v) r[v] = inv_n;
    for (uint32_t t = 0; t < iters; ++t) {
        double dangling = 0.0;
#pragma omp parallel for reduction(+ : dangling) schedule(static)
        for (int64_t u = 0; u < (int64_t)n; ++u) {
            if (outdeg[u]) c[u] = r[u] / (double)outdeg[u];
            else {
                c[u] = 0.0;
                dangling += r[u];
            }
        }
        const double base = (1.0 - damping) * inv_n + damping * dangling * inv_n;
#pragma omp parallel for schedule(dynamic, 4096)
        for (int64_t v = 0; v < (int64_t)n; ++v) {
            double s = 0.0;
            for (uint64_t e = col_ptr[v]; e < col_ptr[v + 1]; ++e) s += c[src[e]];
            r[v] = base + damping * s;
        }
    }
    free(c);
    return 0;
}

/* Min-merge supersteps until quiet: weighted (w != NULL) relaxes d[u] + w
 * (SSSP, INF = 0xFFFFFFFF never relaxed), else takes l[u] (CC). x[n] holds
 * the initial values and receives the result. Returns the supersteps run
 * (including the quiet one), or -1 when scratch cannot be allocated. */
int64_t cb_minlabel_pull(uint64_t n, const uint64_t* col_ptr, const uint32_t* src, const uint32_t* w,
                         uint32_t* x, uint32_t max_steps) {
    uint32_t* y = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!y) return -1;
    int64_t steps = 0;
    for (uint32_t t = 0; t < max_steps; ++t) {
        uint64_t changed = 0;
#pragma omp parallel for reduction(+ : changed) schedule(dynamic, 4096)
        for (int64_t v = 0; v < (int64_t)n; ++v) {
            uint64_t best = x[v];
            for (uint64_t e = col_ptr[v]; e < col_ptr[v + 1]; ++e) {
                const uint32_t xu = x[src[e]];
                if (w) {
                    if (xu == 0xFFFFFFFFu) continue;
                    const uint64_t cand = (uint64_t)xu + w[e];
                    if (cand < best) best = cand;
                } else if (xu < best) {
                    best = xu;
                }
            }
            y[v] = (uint32_t)best;
            changed += best != x[v];
        }
        memcpy(x, y, sizeof(uint32_t) * n);
        ++steps;
        if (!changed) break;
    }
    free(y);
    return steps;
}

/* Binary-heap Dijkstra from `source` over a CSR (row_ptr[n+1] u64, dst[],
 * w[]); dist[n] receives the distances (0xFFFFFFFF unreachable). Returns 0,
 * or -1 when scratch cannot be allocated. */
int cb_dijkstra(uint64_t n, const uint64_t* row_ptr, const uint32_t* dst, const uint32_t* w, uint32_t source,
                uint32_t* dist) {
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
    uint32_t* heap = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t* pos = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!key || !heap || !pos) {
        free(key);
        free(heap);
        free(pos);
        return -1;
    }
    const uint32_t kNone = 0xFFFFFFFFu;
    for (uint64_t v = 0; v < n; ++v) {
        key[v] = UINT64_MAX;
        pos[v] = kNone;
    }
    uint64_t size = 0;
#define CB_SWAP(i, j)                 \
    do {                              \
        uint32_t a_ = heap[i];        \
        heap[i] = heap[j];            \
        heap[j] = a_;                 \
        pos[heap[i]] = (uint32_t)(i); \
        pos[heap[j]] = (uint32_t)(j); \
    } while (0)
    key[source] = 0;
    heap[0] = source;
    pos[source] = 0;
    size = 1;
    while (size) {
        const uint32_t u = heap[0];
        --size;
        pos[u] = kNone - 1u;   /* settled */
        if (size) {
            heap[0] = heap[size];
            pos[heap[0]] = 0;
            uint64_t i = 0;
            for (;;) {
                uint64_t l = 2 * i + 1, r = l + 1, m = i;
                if (l < size && key[heap[l]] < key[heap[m]]) m = l;
                if (r < size && key[heap[r]] < key[heap[m]]) m = r;
                if (m == i) break;
                CB_SWAP(i, m);
                i = m;
            }
        }
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            const uint32_t v = dst[e];
            if (pos[v] == kNone - 1u) continue;
            const uint64_t cand = key[u] + w[e];
            if (cand >= key[v]) continue;
            key[v] = cand;
            uint64_t i;
            if (pos[v] == kNone) {
                i = size++;
                heap[i] = v;
                pos[v] = (uint32_t)i;
            } else {
                i = pos[v];
            }
            while (i > 0) {
                const uint64_t p = (i - 1) / 2;
                if (key[heap[p]] <= key[heap[i]]) break;
                CB_SWAP(i, p);
                i = p;
            }
        }
    }
#undef CB_SWAP
    for (uint64_t v = 0; v < n; ++v) dist[v] = key[v] == UINT64_MAX ? 0xFFFFFFFFu : (uint32_t)key[v];
    free(key);
    free(heap);
    free(pos);
    return 0;
}

static uint32_t cb_find(uint32_t* parent, uint32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];   /* path halving */
        x = parent[x];
    }
    return x;
}

/* Union-find over m edges (src[i], dst[i]); label[n] receives the smallest
 * vertex id of each vertex's component. */
void cb_union_find(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, uint32_t* label) {
    for (uint64_t v = 0; v < n; ++v) label[v] = (uint32_t)v;
    for (uint64_t i = 0; i < m; ++i) {
        const uint32_t a = cb_find(label, src[i]), b = cb_find(label, dst[i]);
        if (a < b) label[b] = a;   /* the smaller id stays the root */
        else if (b < a) label[a] = b;
    }
    for (uint64_t v = 0; v < n; ++v) label[v] = cb_find(label, (uint32_t)v);
}

/* Stable counting sort of m COO edges by destination (one core): col_ptr[n+1]
 * (u64), csrc[m] and, when w != NULL, cw[m]. Returns 0, or -1 when scratch
 * cannot be allocated. */
int cb_csc_build(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, const uint32_t* w,
                 uint64_t* col_ptr, uint32_t* csrc, uint32_t* cw) {
    uint64_t* at = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
    if (!at) return -1;
    memset(col_ptr, 0, sizeof(uint64_t) * (n + 1));
    for (uint64_t i = 0; i < m; ++i) ++col_ptr[dst[i] + 1];
    for (uint64_t v = 0; v < n; ++v) col_ptr[v + 1] += col_ptr[v];
    memcpy(at, col_ptr, sizeof(uint64_t) * n);
    for (uint64_t i = 0; i < m; ++i) {
        const uint64_t k = at[dst[i]]++;
        csrc[k] = src[i];
        if (w) cw[k] = w[i];
    }
    free(at);
    return 0;
}
