/* Route extraction for the synthetic demand generator (input building only).
 *
 * Given shortest-path successor rows pred[row][road] towards a set of
 * destination roads, follow the pointers from each origin until the
 * destination.  mode 0 counts route lengths, mode 1 writes the road sequence
 * at routes[route_off[v] ...].  Returns 0, or -1 when a pointer is missing
 * (unreachable destination) or a walk exceeds max_len.
 */
#include <stdint.h>

int moss_gen_walk(int mode, int64_t n_sel, const int64_t* sel, const int64_t* origins,
                  const int64_t* row_of, const int64_t* dest_of_row, const int32_t* pred,
                  int64_t n_roads, int64_t max_len, int64_t* lengths,
                  const int64_t* route_off, int32_t* routes) {
    for (int64_t k = 0; k < n_sel; ++k) {
        const int64_t v = sel[k];
        const int64_t row = row_of[v];
        const int64_t d = dest_of_row[row];
        const int32_t* p = pred + row * n_roads;
        int64_t cur = origins[v];
        int64_t len = 1;
        int64_t pos = (mode == 1) ? route_off[v] : 0;
        for (;;) {
            if (mode == 1) routes[pos++] = (int32_t)cur;
            if (cur == d) break;
            cur = p[cur];
            if (cur < 0 || ++len > max_len) return -1;
        }
        if (mode == 0) lengths[v] = len;
    }
    return 0;
}

/* Shortest-path successor rows for a set of destinations (input building
 * only).  The road graph is given reversed, in CSR: the edges out of node u
 * are (indices[k], w[k]) for k in [indptr[u], indptr[u+1]), meaning "road
 * indices[k] may be driven just before road u at cost w[k]".  For each
 * destination d = dests[q] a Dijkstra run on the reversed graph gives, for
 * every road v, the next road on a cheapest route from v to d:
 * succ[q * n + v] (-1 if d is unreachable from v, d itself maps to d).
 * Ties in cost are broken by the smaller road id.  Destinations are spread
 * over n_threads POSIX threads; the result does not depend on that number. */
#include <pthread.h>
#include <stdlib.h>

typedef struct {
    int n;
    const int64_t* indptr;
    const int32_t* indices;
    const double* w;
    const int64_t* dests;
    int32_t* succ;
    int q0, q1;
    int rc;
} SuccJob;

typedef struct { double d; int32_t v; } HeapItem;

static int heap_less(HeapItem a, HeapItem b) { return a.d < b.d || (a.d == b.d && a.v < b.v); }

static void heap_push(HeapItem* h, int64_t* sz, HeapItem x) {
    int64_t i = (*sz)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!heap_less(x, h[p])) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = x;
}

static HeapItem heap_pop(HeapItem* h, int64_t* sz) {
    HeapItem top = h[0], x = h[--(*sz)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        HeapItem best = x;
        if (l < *sz && heap_less(h[l], best)) { m = l; best = h[l]; }
        if (r < *sz && heap_less(h[r], best)) { m = r; best = h[r]; }
        if (m == i) break;
        h[i] = h[m];
        i = m;
    }
    h[i] = x;
    return top;
}

static void* succ_worker(void* arg) {
    SuccJob* J = (SuccJob*)arg;
    const int n = J->n;
    double* dist = (double*)malloc(sizeof(double) * (size_t)n);
    char* done = (char*)malloc((size_t)n);
    int64_t cap = (int64_t)J->indptr[n] + n + 1;
    HeapItem* heap = (HeapItem*)malloc(sizeof(HeapItem) * (size_t)cap);
    if (!dist || !done || !heap) { J->rc = -1; free(dist); free(done); free(heap); return NULL; }
    for (int q = J->q0; q < J->q1; ++q) {
        int32_t* succ = J->succ + (int64_t)q * n;
        const int32_t d = (int32_t)J->dests[q];
        for (int v = 0; v < n; ++v) { dist[v] = 1e300; done[v] = 0; succ[v] = -1; }
        int64_t sz = 0;
        dist[d] = 0.0;
        succ[d] = d;
        HeapItem s0 = {0.0, d};
        heap_push(heap, &sz, s0);
        while (sz > 0) {
            HeapItem it = heap_pop(heap, &sz);
            const int32_t u = it.v;
            if (done[u]) continue;
            done[u] = 1;
            for (int64_t k = J->indptr[u]; k < J->indptr[u + 1]; ++k) {
                const int32_t v = J->indices[k];
                const double nd = dist[u] + J->w[k];
                if (nd < dist[v] || (nd == dist[v] && !done[v] && u < succ[v])) {
                    dist[v] = nd;
                    succ[v] = u;
                    HeapItem x = {nd, v};
                    heap_push(heap, &sz, x);
                }
            }
        }
    }
    free(dist); free(done); free(heap);
    J->rc = 0;
    return NULL;
}

int moss_gen_succ(int n, const int64_t* indptr, const int32_t* indices, const double* w, int nd,
                  const int64_t* dests, int32_t* succ, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > nd) n_threads = nd > 0 ? nd : 1;
    SuccJob* jobs = (SuccJob*)calloc((size_t)n_threads, sizeof(SuccJob));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    int rc = 0;
    for (int t = 0; t < n_threads; ++t) {
        jobs[t].n = n; jobs[t].indptr = indptr; jobs[t].indices = indices; jobs[t].w = w;
        jobs[t].dests = dests; jobs[t].succ = succ;
        jobs[t].q0 = (int)((int64_t)nd * t / n_threads);
        jobs[t].q1 = (int)((int64_t)nd * (t + 1) / n_threads);
        if (pthread_create(&th[t], NULL, succ_worker, &jobs[t]) != 0) { jobs[t].rc = -1; th[t] = 0; }
    }
    for (int t = 0; t < n_threads; ++t) {
        if (th[t]) pthread_join(th[t], NULL);
        if (jobs[t].rc != 0) rc = -1;
    }
    free(jobs); free(th);
    return rc;
}
