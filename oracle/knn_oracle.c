/*
 * FP64 brute-force oracle for the PDX search path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * execute this file: only tests/, the smoke check and the bench's CPU
 * baseline do. It shares no code, header or constant with the CUDA library.
 *
 * Every function computes a plain definition, not the PDX algorithm:
 *
 *  - delta()            Sec. 2.1: the squared Euclidean distance
 *                       sum_{j=0}^{D-1} (v_j - q_j)^2 (the paper prints the
 *                       upper limit as D; a D-dimensional vector has indices
 *                       0..D-1), the inner product sum_j v_j q_j (Sec. 2.1 lists
 *                       it among the similarity functions; larger is more
 *                       similar) and the Manhattan distance sum_j |v_j - q_j|.
 *                       The float32 inputs are widened to double before any
 *                       arithmetic.
 *  - oracle_knn()       Sec. 2.1: the k objects that minimise delta (maximise it
 *                       for IP), found by computing delta for every object and
 *                       sorting all of them; ties go to the lower index.
 *  - oracle_knn_probed()  Sec. 2.1 (IVF): the exact top-k restricted to the
 *                       vectors of the nprobe buckets whose centroids are
 *                       nearest to the query (centroid ties: lower bucket id).
 *  - oracle_assign()    Sec. 2.1 (IVF): each vector's nearest centroid.
 *  - oracle_kmeans()    Sec. 2.1 (IVF): Lloyd's algorithm (assign to nearest
 *                       centroid, move each centroid to the mean of its members;
 *                       an empty bucket keeps its centroid), objective per
 *                       iteration.
 *
 * Work is split over queries (or vectors) with pthreads; each thread runs the
 * same plain loops.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { M_L2 = 0, M_IP = 1, M_L1 = 2 };

static double delta(const float *v, const float *q, int32_t d, int32_t metric) {
    double s = 0.0;
    for (int32_t j = 0; j < d; ++j) {
        double a = (double)v[j], b = (double)q[j];
        if (metric == M_L2) s += (a - b) * (a - b);
        else if (metric == M_IP) s += a * b;
        else s += fabs(a - b);
    }
    return s;
}

typedef struct { double key; double d; int64_t i; } ranked_t;

/* Total order: key ascending, then index ascending. key is delta for L2/L1
 * and -delta for IP, so the first k entries are the k best. */
static int cmp_ranked(const void *pa, const void *pb) {
    const ranked_t *a = (const ranked_t *)pa, *b = (const ranked_t *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->i > b->i) - (a->i < b->i);
}

typedef struct {
    const float *x; int64_t n; int32_t d;
    const float *q; int64_t nq; int32_t k; int32_t metric;
    const int32_t *assign; const float *centroids; int32_t nlist; int32_t nprobe;
    double *out_dist; int64_t *out_idx;
    int64_t q0, q1;
    int status;
} knn_job_t;

static void knn_one(const knn_job_t *jb, int64_t qi, ranked_t *buf, ranked_t *cbuf, unsigned char *allowed) {
    const float *q = jb->q + (size_t)qi * jb->d;
    if (jb->assign) {
        for (int32_t c = 0; c < jb->nlist; ++c) {
            double dc = delta(jb->centroids + (size_t)c * jb->d, q, jb->d, M_L2);
            cbuf[c].key = dc; cbuf[c].d = dc; cbuf[c].i = c;
        }
        qsort(cbuf, (size_t)jb->nlist, sizeof(ranked_t), cmp_ranked);
        memset(allowed, 0, (size_t)jb->nlist);
        for (int32_t r = 0; r < jb->nprobe && r < jb->nlist; ++r) allowed[cbuf[r].i] = 1;
    }
    int64_t m = 0;
    for (int64_t i = 0; i < jb->n; ++i) {
        if (jb->assign && !allowed[jb->assign[i]]) continue;
        double dv = delta(jb->x + (size_t)i * jb->d, q, jb->d, jb->metric);
        buf[m].key = (jb->metric == M_IP) ? -dv : dv;
        buf[m].d = dv;
        buf[m].i = i;
        ++m;
    }
    qsort(buf, (size_t)m, sizeof(ranked_t), cmp_ranked);
    for (int32_t r = 0; r < jb->k; ++r) {
        size_t o = (size_t)qi * jb->k + r;
        if (r < m) { jb->out_dist[o] = buf[r].d; jb->out_idx[o] = buf[r].i; }
        else {
            jb->out_dist[o] = (jb->metric == M_IP) ? -INFINITY : INFINITY;
            jb->out_idx[o] = -1;
        }
    }
}

static void *knn_worker(void *arg) {
    knn_job_t *jb = (knn_job_t *)arg;
    ranked_t *buf = (ranked_t *)malloc(sizeof(ranked_t) * (size_t)(jb->n > 0 ? jb->n : 1));
    ranked_t *cbuf = NULL; unsigned char *allowed = NULL;
    if (jb->assign) {
        cbuf = (ranked_t *)malloc(sizeof(ranked_t) * (size_t)jb->nlist);
        allowed = (unsigned char *)malloc((size_t)jb->nlist);
    }
    if (!buf || (jb->assign && (!cbuf || !allowed))) { jb->status = -2; free(buf); free(cbuf); free(allowed); return NULL; }
    for (int64_t qi = jb->q0; qi < jb->q1; ++qi) knn_one(jb, qi, buf, cbuf, allowed);
    free(buf); free(cbuf); free(allowed);
    jb->status = 0;
    return NULL;
}

static int run_knn(knn_job_t base, int32_t nthreads) {
    if (base.d <= 0 || base.k <= 0 || base.n < 0 || base.nq < 0) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > base.nq) nthreads = (int32_t)(base.nq > 0 ? base.nq : 1);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    knn_job_t *jobs = (knn_job_t *)malloc(sizeof(knn_job_t) * (size_t)nthreads);
    if (!th || !jobs) { free(th); free(jobs); return -2; }
    int64_t per = (base.nq + nthreads - 1) / nthreads;
    for (int32_t t = 0; t < nthreads; ++t) {
        jobs[t] = base;
        jobs[t].q0 = (int64_t)t * per;
        jobs[t].q1 = jobs[t].q0 + per < base.nq ? jobs[t].q0 + per : base.nq;
        if (jobs[t].q0 > jobs[t].q1) jobs[t].q0 = jobs[t].q1;
        jobs[t].status = -3;
        pthread_create(&th[t], NULL, knn_worker, &jobs[t]);
    }
    int rc = 0;
    for (int32_t t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].status != 0) rc = jobs[t].status;
    }
    free(th); free(jobs);
    return rc;
}

int oracle_knn(const float *x, int64_t n, int32_t d, const float *q, int64_t nq, int32_t k,
               int32_t metric, int32_t nthreads, double *out_dist, int64_t *out_idx) {
    knn_job_t b;
    memset(&b, 0, sizeof(b));
    b.x = x; b.n = n; b.d = d; b.q = q; b.nq = nq; b.k = k; b.metric = metric;
    b.out_dist = out_dist; b.out_idx = out_idx;
    return run_knn(b, nthreads);
}

int oracle_knn_probed(const float *x, int64_t n, int32_t d, const float *q, int64_t nq, int32_t k,
                      int32_t metric, const int32_t *assign, const float *centroids, int32_t nlist,
                      int32_t nprobe, int32_t nthreads, double *out_dist, int64_t *out_idx) {
    if (!assign || !centroids || nlist <= 0 || nprobe <= 0) return -1;
    knn_job_t b;
    memset(&b, 0, sizeof(b));
    b.x = x; b.n = n; b.d = d; b.q = q; b.nq = nq; b.k = k; b.metric = metric;
    b.assign = assign; b.centroids = centroids; b.nlist = nlist; b.nprobe = nprobe;
    b.out_dist = out_dist; b.out_idx = out_idx;
    return run_knn(b, nthreads);
}

/* ---- nearest centroid and Lloyd iterations ---- */

typedef struct {
    const float *x; int32_t d; const double *c; int32_t nlist;
    int32_t *assign; double *dist; int64_t i0, i1;
} assign_job_t;

static void *assign_worker(void *arg) {
    assign_job_t *a = (assign_job_t *)arg;
    for (int64_t i = a->i0; i < a->i1; ++i) {
        const float *v = a->x + (size_t)i * a->d;
        double best = INFINITY; int32_t bi = -1;
        for (int32_t c = 0; c < a->nlist; ++c) {
            const double *cc = a->c + (size_t)c * a->d;
            double s = 0.0;
            for (int32_t j = 0; j < a->d; ++j) { double t = (double)v[j] - cc[j]; s += t * t; }
            if (s < best) { best = s; bi = c; }   /* strict: ties keep the lower id */
        }
        a->assign[i] = bi;
        if (a->dist) a->dist[i] = best;
    }
    return NULL;
}

static int run_assign(const float *x, int64_t n, int32_t d, const double *c, int32_t nlist,
                      int32_t *assign, double *dist, int32_t nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = (int32_t)(n > 0 ? n : 1);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    assign_job_t *jobs = (assign_job_t *)malloc(sizeof(assign_job_t) * (size_t)nthreads);
    if (!th || !jobs) { free(th); free(jobs); return -2; }
    int64_t per = (n + nthreads - 1) / nthreads;
    for (int32_t t = 0; t < nthreads; ++t) {
        jobs[t].x = x; jobs[t].d = d; jobs[t].c = c; jobs[t].nlist = nlist;
        jobs[t].assign = assign; jobs[t].dist = dist;
        jobs[t].i0 = (int64_t)t * per;
        jobs[t].i1 = jobs[t].i0 + per < n ? jobs[t].i0 + per : n;
        if (jobs[t].i0 > jobs[t].i1) jobs[t].i0 = jobs[t].i1;
        pthread_create(&th[t], NULL, assign_worker, &jobs[t]);
    }
    for (int32_t t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th); free(jobs);
    return 0;
}

int oracle_assign(const float *x, int64_t n, int32_t d, const float *centroids, int32_t nlist,
                  int32_t nthreads, int32_t *out_assign, double *out_dist) {
    if (d <= 0 || nlist <= 0 || n < 0) return -1;
    double *c = (double *)malloc(sizeof(double) * (size_t)nlist * d);
    if (!c) return -2;
    for (size_t i = 0; i < (size_t)nlist * d; ++i) c[i] = (double)centroids[i];
    int rc = run_assign(x, n, d, c, nlist, out_assign, out_dist, nthreads);
    free(c);
    return rc;
}

int oracle_kmeans(const float *x, int64_t n, int32_t d, int32_t nlist, int32_t iters,
                  const float *init_centroids, int32_t nthreads,
                  double *out_centroids, int32_t *out_assign, double *out_objective) {
    if (d <= 0 || nlist <= 0 || n <= 0 || iters < 0) return -1;
    double *c = out_centroids;
    for (size_t i = 0; i < (size_t)nlist * d; ++i) c[i] = (double)init_centroids[i];
    double *dist = (double *)malloc(sizeof(double) * (size_t)n);
    double *sum = (double *)malloc(sizeof(double) * (size_t)nlist * d);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)nlist);
    if (!dist || !sum || !cnt) { free(dist); free(sum); free(cnt); return -2; }
    int rc = 0;
    for (int32_t it = 0; it <= iters; ++it) {
        rc = run_assign(x, n, d, c, nlist, out_assign, dist, nthreads);
        if (rc) break;
        double obj = 0.0;
        for (int64_t i = 0; i < n; ++i) obj += dist[i];
        if (out_objective) out_objective[it] = obj;
        if (it == iters) break;                 /* final assignment only */
        memset(sum, 0, sizeof(double) * (size_t)nlist * d);
        memset(cnt, 0, sizeof(int64_t) * (size_t)nlist);
        for (int64_t i = 0; i < n; ++i) {
            int32_t a = out_assign[i];
            cnt[a] += 1;
            for (int32_t j = 0; j < d; ++j) sum[(size_t)a * d + j] += (double)x[(size_t)i * d + j];
        }
        for (int32_t a = 0; a < nlist; ++a) {
            if (cnt[a] == 0) continue;          /* empty bucket keeps its centroid */
            for (int32_t j = 0; j < d; ++j) c[(size_t)a * d + j] = sum[(size_t)a * d + j] / (double)cnt[a];
        }
    }
    free(dist); free(sum); free(cnt);
    return rc;
}
