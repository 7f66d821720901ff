/*
 * tmfg_oracle.c -- plain, slow, single-purpose CPU oracle for the TMFG-DBHT
 * hot path of Raphael & Shun, "Faster Parallel Triangular Maximally Filtered
 * Graphs and Hierarchical Clustering" (arXiv 2408.09399).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is built into oracle/liboracle.so and
 * is loaded by the test-suite, by the smoke check and by the CPU-baseline leg
 * of the benchmark.  The CUDA library never links, includes or calls it, and
 * it shares no source with the CUDA library.
 *
 * What it follows:
 *   - Algorithm 1 (corr-tmfg, Section 4.1) and Algorithm 2 (heap-tmfg,
 *     Section 4.2): initial 4-clique from row sums, one up-front sort of
 *     every row of S, MaxCorrs as the best uninserted vertex of a row, face
 *     candidates V_m[f], the Gains array / max-heap, insertion of a vertex
 *     into a face (3 edges, 3 faces replacing 1).
 *   - Section 4.3: the lazily advanced pointer into each sorted row and the
 *     hub-based approximate all-pairs shortest paths.
 *   - Section 2 (PMFG, TMFG and DBHT): the exact greedy TMFG (Massara et al.),
 *     APSP by one Dijkstra per source, and the DBHT bubble tree, edge
 *     directions, converging bubbles, vertex assignment and three-level
 *     complete linkage.
 *   - Section 5 (Evaluation): the adjusted Rand index and the cut of the
 *     dendrogram at k clusters.
 *
 * Readings taken where the paper is silent (the CUDA path takes the same):
 *   R1  S is read as given: row v of the sort is S[v,*]; the gain of vertex u
 *       for face {a<b<c} is (S[a,u] + S[b,u]) + S[c,u], summed in that order
 *       in the input precision (float or double), round-to-nearest, no FMA.
 *       -0.0 is the same similarity as +0.0.  The diagonal is never used.
 *   R2  Row sum r_v = sum over u != v of q(S[v,u]), q(x) = x*2^40 rounded to
 *       the nearest integer (ties to even), summed exactly in int64.  The
 *       initial clique v1..v4 is the top four by (r desc, id asc).
 *   R3  Row v sorted by (S[v,u] desc, u asc) over u != v.
 *   R4  MaxCorrs[w] is read fresh: the first uninserted vertex of row w's
 *       sorted order (the lazily advanced pointer of Section 4.3).
 *   R5  Best vertex of a face: among the distinct MaxCorrs of its three
 *       vertices, max gain, ties to the smaller vertex id.
 *   R6  A face-vertex pair ranks by (gain desc, vertex asc, face id asc).
 *   R7  Face ids: faces 0..3 are {v1,v2,v3},{v1,v2,v4},{v1,v3,v4},{v2,v3,v4};
 *       inserting v into face t={x<y<z} puts {v,x,y} into slot t and appends
 *       {v,y,z} then {v,x,z}; every face is stored with its ids ascending.
 *   R8  corr-tmfg: L = the P best pairs by R6; keep the first pair per vertex;
 *       insert in rank order; then recompute exactly the faces whose stored
 *       vertex was inserted this round plus the new faces (F_update).
 *   R9  heap-tmfg: a binary max-heap ordered by R6 with one entry per face.
 *   R10 Bubble 0 is the initial clique, bubble k is the k-th insertion
 *       {v_k} + t_k; its parent is the bubble that created face t_k.
 *   R11 Edge length sqrt(max(0, 2(1 - S[a,b]))) for TMFG edge (a,b).
 *   R12 Approximate APSP: hubs are the ceil(sqrt n) vertices of largest
 *       degree (ties to the smaller id); h(s) the nearest hub (ties to the
 *       lower hub rank) at distance d_s; radius r_s = rf * d_s;
 *       D[s,t] = min(d_s + D(h(s),t), d_t + D(h(t),s), and the exact
 *       distance from s if it is <= r_s, and from t if it is <= r_t).
 *   R13 DBHT: see oracle_dbht below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_F32 0
#define OR_F64 1
#define OR_NONE (-1)

#define OR_CORR 0
#define OR_HEAP 1

/* return codes */
#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

/* Host threads used by the parallel loops (rows of the sort, sources of
 * the APSP); k < 1 leaves the setting alone.  Returns the number in use. */
int oracle_set_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
    return omp_get_max_threads();
#else
    (void)k;
    return 1;
#endif
}

/* Monotonic clock in nanoseconds (phase timings of oracle_tmfg). */
static int64_t now_ns(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000 + ts.tv_nsec;
}

/* ------------------------------------------------------------------ */
/* matrix access                                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    const void *S;
    int64_t n, ld;
    int dtype;
} mat_t;

/* S[i,j] as a double (exact for float input); -0.0 is returned as +0.0. */
static double sget(const mat_t *m, int64_t i, int64_t j)
{
    double x;
    if (m->dtype == OR_F32)
        x = (double)((const float *)m->S)[i * m->ld + j];
    else
        x = ((const double *)m->S)[i * m->ld + j];
    return x == 0.0 ? 0.0 : x;
}

/* Gain of vertex u for face {x<y<z} in the input precision (R1).  A float
 * sum is returned widened to double, which is exact and keeps the order. */
static double face_gain(const mat_t *m, int32_t x, int32_t y, int32_t z, int32_t u)
{
    if (m->dtype == OR_F32) {
        float a = (float)sget(m, x, u);
        float b = (float)sget(m, y, u);
        float c = (float)sget(m, z, u);
        float s = a + b;
        s = s + c;
        return (double)s;
    } else {
        double s = sget(m, x, u) + sget(m, y, u);
        s = s + sget(m, z, u);
        return s;
    }
}

/* 1 if pair (g1,v1,f1) ranks strictly above (g2,v2,f2) under R6. */
static int ranks_above(double g1, int32_t v1, int32_t f1, double g2, int32_t v2, int32_t f2)
{
    if (g1 != g2) return g1 > g2;
    if (v1 != v2) return v1 < v2;
    return f1 < f2;
}

/* ------------------------------------------------------------------ */
/* row sums and the initial clique (Algorithm 1, first lines; R2)        */
/* ------------------------------------------------------------------ */

int64_t oracle_quantize(double x)
{
    return llrint(x * 1099511627776.0); /* 2^40, default rounding = nearest-even */
}

void oracle_rowsums(const void *S, int64_t n, int64_t ld, int dtype, int64_t *rowsum)
{
    mat_t m = {S, n, ld, dtype};
    for (int64_t v = 0; v < n; ++v) {
        int64_t r = 0;
        for (int64_t u = 0; u < n; ++u)
            if (u != v) r += oracle_quantize(sget(&m, v, u));
        rowsum[v] = r;
    }
}

/* top four by (r desc, id asc), written in rank order */
static void pick_clique(const int64_t *r, int64_t n, int32_t out[4])
{
    for (int k = 0; k < 4; ++k) {
        int32_t best = OR_NONE;
        for (int64_t v = 0; v < n; ++v) {
            int taken = 0;
            for (int j = 0; j < k; ++j) taken |= (out[j] == v);
            if (taken) continue;
            if (best == OR_NONE || r[v] > r[best]) best = (int32_t)v;
        }
        out[k] = best;
    }
}

/* ------------------------------------------------------------------ */
/* per-row sort (Algorithm 1, sort loop; R3)                             */
/* ------------------------------------------------------------------ */

typedef struct {
    double s;
    int32_t u;
} su_t;

static int cmp_su(const void *pa, const void *pb)
{
    const su_t *a = (const su_t *)pa, *b = (const su_t *)pb;
    if (a->s != b->s) return a->s > b->s ? -1 : 1;
    return (a->u > b->u) - (a->u < b->u);
}

/* idx: n rows of n-1 entries (row-major, stride n-1). */
int oracle_rowsort(const void *S, int64_t n, int64_t ld, int dtype, int32_t *idx)
{
    if (n < 2) return OR_EINVAL;
    mat_t m = {S, n, ld, dtype};
    int rc = OR_OK;
#pragma omp parallel
    {
        su_t *buf = (su_t *)malloc(sizeof(su_t) * (size_t)n);
        if (!buf) {
#pragma omp atomic write
            rc = OR_ENOMEM;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t v = 0; v < n; ++v) {
            if (!buf) continue;
            int64_t k = 0;
            for (int64_t u = 0; u < n; ++u)
                if (u != v) {
                    buf[k].s = sget(&m, v, u);
                    buf[k].u = (int32_t)u;
                    ++k;
                }
            qsort(buf, (size_t)k, sizeof(su_t), cmp_su);
            for (int64_t j = 0; j < k; ++j) idx[v * (n - 1) + j] = buf[j].u;
        }
        free(buf);
    }
    return rc;
}

/* ------------------------------------------------------------------ */
/* TMFG state shared by corr-tmfg, heap-tmfg and the exact greedy        */
/* ------------------------------------------------------------------ */

typedef struct {
    mat_t m;
    int64_t n;
    const int32_t *idx; /* sorted rows, stride n-1 (NULL for the exact greedy) */
    int64_t *ptr;       /* lazy pointer per row (R4) */
    int mc_bruteforce;  /* 1: MaxCorrs by a full argmax instead of the pointer */
    uint8_t *inserted;
    int64_t nrem;
    /* faces */
    int32_t *fa, *fb, *fc; /* ascending ids */
    int32_t *fv;           /* stored best vertex (OR_NONE if no candidate) */
    double *fg;            /* stored gain */
    int32_t *fown;         /* bubble that created the face */
    int64_t nf;
    /* outputs */
    int32_t *order, *edges, *ins_face, *parent;
    double *ins_gain; /* optional: gain of each inserted pair */
    int64_t k;        /* insertions done */
    /* counters */
    int64_t face_evals, stale_pops;
} tstate;

static void sort3(int32_t *a, int32_t *b, int32_t *c)
{
    int32_t t;
    if (*a > *b) { t = *a; *a = *b; *b = t; }
    if (*b > *c) { t = *b; *b = *c; *c = t; }
    if (*a > *b) { t = *a; *a = *b; *b = t; }
}

static void set_face(tstate *st, int64_t f, int32_t a, int32_t b, int32_t c, int32_t owner)
{
    sort3(&a, &b, &c);
    st->fa[f] = a;
    st->fb[f] = b;
    st->fc[f] = c;
    st->fv[f] = OR_NONE;
    st->fg[f] = -INFINITY;
    st->fown[f] = owner;
}

/* MaxCorrs[w]: best uninserted vertex of row w (R4), or OR_NONE. */
static int32_t maxcorrs(tstate *st, int32_t w)
{
    int64_t n = st->n;
    if (st->mc_bruteforce) {
        int32_t best = OR_NONE;
        double bs = 0.0;
        for (int64_t u = 0; u < n; ++u) {
            if (u == w || st->inserted[u]) continue;
            double s = sget(&st->m, w, u);
            if (best == OR_NONE || s > bs) { best = (int32_t)u; bs = s; }
        }
        return best;
    }
    const int32_t *row = st->idx + (int64_t)w * (n - 1);
    while (st->ptr[w] < n - 1 && st->inserted[row[st->ptr[w]]]) st->ptr[w]++;
    return st->ptr[w] < n - 1 ? row[st->ptr[w]] : OR_NONE;
}

/* Recompute the stored best vertex of face f from fresh MaxCorrs (R5). */
static void face_best(tstate *st, int64_t f)
{
    int32_t x = st->fa[f], y = st->fb[f], z = st->fc[f];
    int32_t cand[3] = {maxcorrs(st, x), maxcorrs(st, y), maxcorrs(st, z)};
    int32_t bv = OR_NONE;
    double bg = -INFINITY;
    for (int i = 0; i < 3; ++i) {
        int32_t u = cand[i];
        if (u == OR_NONE) continue;
        double g = face_gain(&st->m, x, y, z, u);
        if (bv == OR_NONE || g > bg || (g == bg && u < bv)) { bv = u; bg = g; }
    }
    st->fv[f] = bv;
    st->fg[f] = bg;
    st->face_evals++;
}

/* Insert vertex v into face f (R7, R10); returns the ids of the 3 new faces. */
static void insert_pair(tstate *st, int32_t v, int64_t f, double g, int64_t newf[3])
{
    int64_t k = st->k;
    int32_t x = st->fa[f], y = st->fb[f], z = st->fc[f];
    st->order[4 + k] = v;
    st->edges[2 * (6 + 3 * k) + 0] = v; st->edges[2 * (6 + 3 * k) + 1] = x;
    st->edges[2 * (6 + 3 * k) + 2] = v; st->edges[2 * (6 + 3 * k) + 3] = y;
    st->edges[2 * (6 + 3 * k) + 4] = v; st->edges[2 * (6 + 3 * k) + 5] = z;
    st->ins_face[3 * k + 0] = x;
    st->ins_face[3 * k + 1] = y;
    st->ins_face[3 * k + 2] = z;
    st->parent[k + 1] = st->fown[f];
    if (st->ins_gain) st->ins_gain[k] = g;
    int32_t bub = (int32_t)(k + 1);
    set_face(st, f, v, x, y, bub);
    set_face(st, st->nf, v, y, z, bub);
    set_face(st, st->nf + 1, v, x, z, bub);
    newf[0] = f;
    newf[1] = st->nf;
    newf[2] = st->nf + 1;
    st->nf += 2;
    st->inserted[v] = 1;
    st->nrem--;
    st->k++;
}

static void tstate_free(tstate *st)
{
    free(st->ptr); free(st->inserted);
    free(st->fa); free(st->fb); free(st->fc); free(st->fv); free(st->fg); free(st->fown);
}

static int tstate_init(tstate *st, const void *S, int64_t n, int64_t ld, int dtype,
                       int32_t *order, int32_t *edges, int32_t *ins_face, int32_t *parent,
                       double *ins_gain, int64_t *rowsum_out)
{
    memset(st, 0, sizeof(*st));
    st->m.S = S; st->m.n = n; st->m.ld = ld; st->m.dtype = dtype;
    st->n = n;
    int64_t nfmax = 2 * n - 4;
    st->ptr = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    st->inserted = (uint8_t *)calloc((size_t)n, 1);
    st->fa = (int32_t *)malloc(sizeof(int32_t) * nfmax);
    st->fb = (int32_t *)malloc(sizeof(int32_t) * nfmax);
    st->fc = (int32_t *)malloc(sizeof(int32_t) * nfmax);
    st->fv = (int32_t *)malloc(sizeof(int32_t) * nfmax);
    st->fg = (double *)malloc(sizeof(double) * nfmax);
    st->fown = (int32_t *)malloc(sizeof(int32_t) * nfmax);
    int64_t *r = (int64_t *)malloc(sizeof(int64_t) * n);
    if (!st->ptr || !st->inserted || !st->fa || !st->fb || !st->fc || !st->fv || !st->fg ||
        !st->fown || !r) {
        free(r);
        tstate_free(st);
        return OR_ENOMEM;
    }
    st->order = order; st->edges = edges; st->ins_face = ins_face; st->parent = parent;
    st->ins_gain = ins_gain;

    /* initial 4-clique (R2) */
    oracle_rowsums(S, n, ld, dtype, r);
    if (rowsum_out) memcpy(rowsum_out, r, sizeof(int64_t) * n);
    int32_t c[4];
    pick_clique(r, n, c);
    free(r);
    for (int i = 0; i < 4; ++i) { order[i] = c[i]; st->inserted[c[i]] = 1; }
    /* edges in the order of Algorithm 1 */
    int32_t e0[6][2] = {{c[0], c[1]}, {c[0], c[2]}, {c[0], c[3]},
                        {c[1], c[2]}, {c[1], c[3]}, {c[2], c[3]}};
    for (int i = 0; i < 6; ++i) { edges[2 * i] = e0[i][0]; edges[2 * i + 1] = e0[i][1]; }
    set_face(st, 0, c[0], c[1], c[2], 0);
    set_face(st, 1, c[0], c[1], c[3], 0);
    set_face(st, 2, c[0], c[2], c[3], 0);
    set_face(st, 3, c[1], c[2], c[3], 0);
    st->nf = 4;
    parent[0] = -1;
    st->nrem = n - 4;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* corr-tmfg (Algorithm 1; R8)                                           */
/* ------------------------------------------------------------------ */

static int run_corr(tstate *st, int64_t P)
{
    int64_t nfmax = 2 * st->n - 4;
    int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (size_t)P);
    uint8_t *picked = (uint8_t *)calloc((size_t)nfmax, 1);
    uint8_t *round_ins = (uint8_t *)calloc((size_t)st->n, 1);
    uint8_t *is_new = (uint8_t *)calloc((size_t)nfmax, 1);
    int32_t *kept_v = (int32_t *)malloc(sizeof(int32_t) * (size_t)P);
    int64_t *kept_f = (int64_t *)malloc(sizeof(int64_t) * (size_t)P);
    if (!L || !picked || !round_ins || !is_new || !kept_v || !kept_f) {
        free(L); free(picked); free(round_ins); free(is_new); free(kept_v); free(kept_f);
        return OR_ENOMEM;
    }
    for (int64_t f = 0; f < st->nf; ++f) face_best(st, f);

    while (st->nrem > 0) {
        /* L: the P best pairs of the Gains array (by repeated argmax) */
        int64_t nl = 0;
        while (nl < P && nl < st->nf) {
            int64_t bf = -1;
            for (int64_t f = 0; f < st->nf; ++f) {
                if (picked[f] || st->fv[f] == OR_NONE) continue;
                if (bf < 0 || ranks_above(st->fg[f], st->fv[f], (int32_t)f,
                                          st->fg[bf], st->fv[bf], (int32_t)bf))
                    bf = f;
            }
            if (bf < 0) break;
            picked[bf] = 1;
            L[nl++] = bf;
        }
        /* keep only the best pair of each vertex */
        int64_t nk = 0;
        for (int64_t i = 0; i < nl; ++i) {
            int32_t v = st->fv[L[i]];
            int dup = 0;
            for (int64_t j = 0; j < nk; ++j) dup |= (kept_v[j] == v);
            if (!dup) { kept_v[nk] = v; kept_f[nk] = L[i]; ++nk; }
        }
        for (int64_t i = 0; i < nl; ++i) picked[L[i]] = 0;
        int bad = (nk == 0);
        for (int64_t i = 0; i < nk; ++i) bad |= st->inserted[kept_v[i]];
        if (bad) { /* every stored vertex is uninserted after F_update */
            free(L); free(picked); free(round_ins); free(is_new); free(kept_v); free(kept_f);
            return OR_EINVAL;
        }
        /* insert in rank order */
        for (int64_t i = 0; i < nk; ++i) {
            int64_t nf3[3];
            round_ins[kept_v[i]] = 1;
            insert_pair(st, kept_v[i], kept_f[i], st->fg[kept_f[i]], nf3);
            for (int j = 0; j < 3; ++j) is_new[nf3[j]] = 1;
        }
        /* F_update: new faces and faces whose stored vertex was inserted */
        for (int64_t f = 0; f < st->nf; ++f) {
            if (is_new[f] || (st->fv[f] != OR_NONE && round_ins[st->fv[f]])) {
                face_best(st, f);
                is_new[f] = 0;
            }
        }
        for (int64_t i = 0; i < nk; ++i) round_ins[kept_v[i]] = 0;
    }
    free(L); free(picked); free(round_ins); free(is_new); free(kept_v); free(kept_f);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* heap-tmfg (Algorithm 2; R9)                                           */
/* ------------------------------------------------------------------ */

typedef struct {
    double g;
    int32_t v;
    int32_t f;
} hent_t;

static int hent_above(const hent_t *a, const hent_t *b)
{
    return ranks_above(a->g, a->v, a->f, b->g, b->v, b->f);
}

static void heap_push(hent_t *h, int64_t *sz, hent_t e)
{
    int64_t i = (*sz)++;
    h[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!hent_above(&h[i], &h[p])) break;
        hent_t t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static hent_t heap_pop(hent_t *h, int64_t *sz)
{
    hent_t top = h[0];
    h[0] = h[--(*sz)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, b = i;
        if (l < *sz && hent_above(&h[l], &h[b])) b = l;
        if (r < *sz && hent_above(&h[r], &h[b])) b = r;
        if (b == i) break;
        hent_t t = h[i]; h[i] = h[b]; h[b] = t;
        i = b;
    }
    return top;
}

static hent_t face_entry(const tstate *st, int64_t f)
{
    hent_t e = {st->fg[f], st->fv[f], (int32_t)f};
    return e;
}

static int run_heap(tstate *st)
{
    int64_t nfmax = 2 * st->n - 4;
    hent_t *h = (hent_t *)malloc(sizeof(hent_t) * (size_t)nfmax);
    if (!h) return OR_ENOMEM;
    int64_t sz = 0;
    for (int64_t f = 0; f < st->nf; ++f) {
        face_best(st, f);
        heap_push(h, &sz, face_entry(st, f));
    }
    while (st->nrem > 0 && sz > 0) {
        hent_t e = heap_pop(h, &sz);
        if (e.v == OR_NONE) continue; /* cannot happen while vertices remain */
        if (st->inserted[e.v]) {
            /* stale pair: recompute this face only and push it back */
            st->stale_pops++;
            face_best(st, e.f);
            if (st->fv[e.f] != OR_NONE && st->inserted[st->fv[e.f]]) {
                free(h); /* a fresh MaxCorrs is never an inserted vertex */
                return OR_EINVAL;
            }
            heap_push(h, &sz, face_entry(st, e.f));
        } else {
            int64_t nf3[3];
            insert_pair(st, e.v, e.f, e.g, nf3);
            for (int j = 0; j < 3; ++j) {
                face_best(st, nf3[j]);
                heap_push(h, &sz, face_entry(st, nf3[j]));
            }
        }
    }
    free(h);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* exact greedy TMFG (Massara et al.; the P=1 orig-tmfg of Section 2)    */
/* ------------------------------------------------------------------ */

static void run_exact_greedy(tstate *st)
{
    while (st->nrem > 0) {
        int64_t bf = -1;
        int32_t bu = OR_NONE;
        double bg = -INFINITY;
        for (int64_t f = 0; f < st->nf; ++f)
            for (int64_t u = 0; u < st->n; ++u) {
                if (st->inserted[u]) continue;
                double g = face_gain(&st->m, st->fa[f], st->fb[f], st->fc[f], (int32_t)u);
                if (bf < 0 || ranks_above(g, (int32_t)u, (int32_t)f, bg, bu, (int32_t)bf)) {
                    bf = f; bu = (int32_t)u; bg = g;
                }
            }
        int64_t nf3[3];
        insert_pair(st, bu, bf, bg, nf3);
    }
}

/* ------------------------------------------------------------------ */
/* public TMFG entry point                                              */
/* ------------------------------------------------------------------ */

/* mode: OR_CORR (with prefix P >= 1) or OR_HEAP (P must be 1), or 2 for
 * the exact greedy.  flags bit 0: MaxCorrs by brute-force argmax.
 * Outputs: order[n], edges[(3n-6)*2], ins_face[(n-4)*3], parent[n-3];
 * optional: ins_gain[n-4], rowsum[n], final faces faces[(2n-4)*3],
 * stats[2] = {face evaluations, stale heap pops}. */
int oracle_tmfg(const void *S, int64_t n, int64_t ld, int dtype, int mode, int64_t P, int flags,
                int32_t *order, int32_t *edges, int32_t *ins_face, int32_t *parent,
                double *ins_gain, int64_t *rowsum, int32_t *faces, int64_t *stats)
{
    if (n < 4 || ld < n || (dtype != OR_F32 && dtype != OR_F64)) return OR_EINVAL;
    if (mode == OR_CORR && P < 1) return OR_EINVAL;
    if (mode == OR_HEAP && P != 1) return OR_EINVAL;
    if (mode != OR_CORR && mode != OR_HEAP && mode != 2) return OR_EINVAL;
    tstate st;
    const int64_t t0 = now_ns();
    int rc = tstate_init(&st, S, n, ld, dtype, order, edges, ins_face, parent, ins_gain, rowsum);
    if (rc) return rc;
    const int64_t t1 = now_ns();
    int32_t *idx = NULL;
    if (mode != 2 && !(flags & 1)) {
        idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)(n - 1));
        if (!idx) { tstate_free(&st); return OR_ENOMEM; }
        rc = oracle_rowsort(S, n, ld, dtype, idx);
        if (rc) { free(idx); tstate_free(&st); return rc; }
    }
    const int64_t t2 = now_ns();
    st.idx = idx;
    st.mc_bruteforce = (flags & 1);
    if (mode == OR_CORR) rc = run_corr(&st, P);
    else if (mode == OR_HEAP) rc = run_heap(&st);
    else run_exact_greedy(&st);
    const int64_t t3 = now_ns();
    if (faces)
        for (int64_t f = 0; f < st.nf; ++f) {
            faces[3 * f] = st.fa[f]; faces[3 * f + 1] = st.fb[f]; faces[3 * f + 2] = st.fc[f];
        }
    /* stats: face evaluations, stale pops, then the wall time (ns) of the
       row sums + initial clique, the row sort and the insertion loop */
    if (stats) {
        stats[0] = st.face_evals; stats[1] = st.stale_pops;
        stats[2] = t1 - t0; stats[3] = t2 - t1; stats[4] = t3 - t2;
    }
    free(idx);
    tstate_free(&st);
    return rc;
}

/* ------------------------------------------------------------------ */
/* APSP over the TMFG (Section 2: one Dijkstra per source; R11)          */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    int64_t *rowptr; /* n+1 */
    int32_t *col;
    double *len;     /* precision-rounded length (float lengths stored widened) */
} graph_t;

static void graph_free(graph_t *g) { free(g->rowptr); free(g->col); free(g->len); }

/* Edge length of TMFG edge (a,b) from S[a,b] (R11).  prec 32: computed in
 * the input precision and rounded to float, as the FP32 distance path
 * does; prec 64: computed in double from the stored value. */
static double edge_len(const mat_t *m, int32_t a, int32_t b, int prec)
{
    double s = sget(m, a, b);
    if (prec == 64) {
        double t = 2.0 * (1.0 - s);
        return sqrt(t > 0.0 ? t : 0.0);
    }
    if (m->dtype == OR_F32) {
        float sf = (float)s;
        float t = 1.0f - sf;
        t = 2.0f * t;
        return (double)sqrtf(t > 0.0f ? t : 0.0f);
    } else {
        double t = 2.0 * (1.0 - s);
        return (double)(float)sqrt(t > 0.0 ? t : 0.0);
    }
}

static int build_graph(const mat_t *m, int64_t n, const int32_t *edges, int64_t ne, int prec,
                       graph_t *g)
{
    g->n = n;
    g->rowptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * ne));
    g->len = (double *)malloc(sizeof(double) * (size_t)(2 * ne));
    int64_t *fill = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    if (!g->rowptr || !g->col || !g->len || !fill) { free(fill); graph_free(g); return OR_ENOMEM; }
    for (int64_t e = 0; e < ne; ++e) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) { free(fill); graph_free(g); return OR_EINVAL; }
        g->rowptr[a + 1]++;
        g->rowptr[b + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) g->rowptr[v + 1] += g->rowptr[v];
    for (int64_t e = 0; e < ne; ++e) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        double l = edge_len(m, a, b, prec);
        int64_t pa = g->rowptr[a] + fill[a]++, pb = g->rowptr[b] + fill[b]++;
        g->col[pa] = b; g->len[pa] = l;
        g->col[pb] = a; g->len[pb] = l;
    }
    free(fill);
    return OR_OK;
}

typedef struct {
    double d;
    int32_t v;
} dent_t;

static void dheap_push(dent_t *h, int64_t *sz, dent_t e)
{
    int64_t i = (*sz)++;
    h[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d <= h[i].d) break;
        dent_t t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static dent_t dheap_pop(dent_t *h, int64_t *sz)
{
    dent_t top = h[0];
    h[0] = h[--(*sz)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, b = i;
        if (l < *sz && h[l].d < h[b].d) b = l;
        if (r < *sz && h[r].d < h[b].d) b = r;
        if (b == i) break;
        dent_t t = h[i]; h[i] = h[b]; h[b] = t;
        i = b;
    }
    return top;
}

/* Dijkstra from src.  prec 32: every tentative distance is a float sum
 * dist[u] + len (the distance along a path is the left-to-right float sum of
 * its lengths, minimised over paths).  bound >= 0: vertices whose distance
 * exceeds bound are not expanded (their dist stays as found or +inf).
 * dist[] and work buffers are caller-owned. */
static void dijkstra(const graph_t *g, int32_t src, int prec, double bound, double *dist,
                     uint8_t *done, dent_t *heap)
{
    int64_t n = g->n, sz = 0;
    for (int64_t v = 0; v < n; ++v) { dist[v] = INFINITY; done[v] = 0; }
    dist[src] = 0.0;
    dent_t s0 = {0.0, src};
    dheap_push(heap, &sz, s0);
    while (sz > 0) {
        dent_t e = dheap_pop(heap, &sz);
        if (done[e.v]) continue;
        if (e.d != dist[e.v]) continue;
        done[e.v] = 1;
        if (bound >= 0.0 && e.d > bound) continue;
        for (int64_t p = g->rowptr[e.v]; p < g->rowptr[e.v + 1]; ++p) {
            int32_t w = g->col[p];
            double nd;
            if (prec == 32) nd = (double)((float)e.d + (float)g->len[p]);
            else nd = e.d + g->len[p];
            if (nd < dist[w]) {
                dist[w] = nd;
                dent_t ne = {nd, w};
                dheap_push(heap, &sz, ne);
            }
        }
    }
}

/* D: n x n doubles (row-major).  edges: (3n-6) x 2.  prec: 32 or 64. */
int oracle_apsp_exact(const void *S, int64_t n, int64_t ld, int dtype, const int32_t *edges,
                      int64_t ne, int prec, double *D)
{
    if (n < 1 || (prec != 32 && prec != 64)) return OR_EINVAL;
    mat_t m = {S, n, ld, dtype};
    graph_t g;
    int rc = build_graph(&m, n, edges, ne, prec, &g);
    if (rc) return rc;
#pragma omp parallel
    {
        uint8_t *done = (uint8_t *)malloc((size_t)n);
        dent_t *heap = (dent_t *)malloc(sizeof(dent_t) * (size_t)(2 * ne + n + 1));
#pragma omp for schedule(dynamic, 8)
        for (int64_t s = 0; s < n; ++s)
            if (done && heap) dijkstra(&g, (int32_t)s, prec, -1.0, D + s * n, done, heap);
        if (!done || !heap) {
#pragma omp atomic write
            rc = OR_ENOMEM;
        }
        free(done);
        free(heap);
    }
    graph_free(&g);
    return rc;
}

/* Exact SSSP rows for a list of sources only (used for sampled checks). */
int oracle_sssp_rows(const void *S, int64_t n, int64_t ld, int dtype, const int32_t *edges,
                     int64_t ne, int prec, const int32_t *src, int64_t nsrc, double *D)
{
    if (n < 1 || (prec != 32 && prec != 64)) return OR_EINVAL;
    mat_t m = {S, n, ld, dtype};
    graph_t g;
    int rc = build_graph(&m, n, edges, ne, prec, &g);
    if (rc) return rc;
#pragma omp parallel
    {
        uint8_t *done = (uint8_t *)malloc((size_t)n);
        dent_t *heap = (dent_t *)malloc(sizeof(dent_t) * (size_t)(2 * ne + n + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < nsrc; ++i)
            if (done && heap) dijkstra(&g, src[i], prec, -1.0, D + i * n, done, heap);
        if (!done || !heap) {
#pragma omp atomic write
            rc = OR_ENOMEM;
        }
        free(done); free(heap);
    }
    graph_free(&g);
    return rc;
}

/* Bounded searches: for each listed source, Dijkstra that does not expand
 * vertices farther than bound[i] (the radius search of Section 4.3).  Row i
 * of D holds the distances found (exact for every vertex within the bound). */
int oracle_sssp_bounded_rows(const void *S, int64_t n, int64_t ld, int dtype,
                             const int32_t *edges, int64_t ne, int prec, const int32_t *src,
                             const double *bound, int64_t nsrc, double *D)
{
    if (n < 1 || (prec != 32 && prec != 64)) return OR_EINVAL;
    mat_t m = {S, n, ld, dtype};
    graph_t g;
    int rc = build_graph(&m, n, edges, ne, prec, &g);
    if (rc) return rc;
#pragma omp parallel
    {
        uint8_t *done = (uint8_t *)malloc((size_t)n);
        dent_t *heap = (dent_t *)malloc(sizeof(dent_t) * (size_t)(2 * ne + n + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < nsrc; ++i)
            if (done && heap) dijkstra(&g, src[i], prec, bound[i], D + i * n, done, heap);
        if (!done || !heap) {
#pragma omp atomic write
            rc = OR_ENOMEM;
        }
        free(done); free(heap);
    }
    graph_free(&g);
    return rc;
}

/* Rows of the per-row sort for the listed rows only (same order as R3). */
int oracle_rowsort_rows(const void *S, int64_t n, int64_t ld, int dtype, const int32_t *rows,
                        int64_t nrows, int32_t *idx)
{
    if (n < 2) return OR_EINVAL;
    mat_t m = {S, n, ld, dtype};
    su_t *buf = (su_t *)malloc(sizeof(su_t) * (size_t)n);
    if (!buf) return OR_ENOMEM;
    for (int64_t i = 0; i < nrows; ++i) {
        int64_t v = rows[i], k = 0;
        for (int64_t u = 0; u < n; ++u)
            if (u != v) { buf[k].s = sget(&m, v, u); buf[k].u = (int32_t)u; ++k; }
        qsort(buf, (size_t)k, sizeof(su_t), cmp_su);
        for (int64_t j = 0; j < k; ++j) idx[i * (n - 1) + j] = buf[j].u;
    }
    free(buf);
    return OR_OK;
}

/* Hubs (R12): the h vertices of largest TMFG degree, ties to the smaller id,
 * listed in that rank order. */
int oracle_hubs(int64_t n, const int32_t *edges, int64_t ne, int64_t h, int32_t *hubs)
{
    if (h < 1 || h > n) return OR_EINVAL;
    int64_t *deg = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    uint8_t *taken = (uint8_t *)calloc((size_t)n, 1);
    if (!deg || !taken) { free(deg); free(taken); return OR_ENOMEM; }
    for (int64_t e = 0; e < ne; ++e) { deg[edges[2 * e]]++; deg[edges[2 * e + 1]]++; }
    for (int64_t i = 0; i < h; ++i) {
        int64_t b = -1;
        for (int64_t v = 0; v < n; ++v)
            if (!taken[v] && (b < 0 || deg[v] > deg[b])) b = v;
        taken[b] = 1;
        hubs[i] = (int32_t)b;
    }
    free(deg); free(taken);
    return OR_OK;
}

/* Approximate APSP (Section 4.3; reading R12).  h = n_hubs (0: ceil(sqrt n)),
 * rf = radius factor (<= 0: 2).  Arithmetic in prec 32 (float) or 64.
 * Optional outputs: hubs[h], nearest[n] (hub rank of h(s)), dnear[n] (d_s). */
int oracle_apsp_approx(const void *S, int64_t n, int64_t ld, int dtype, const int32_t *edges,
                       int64_t ne, int64_t n_hubs, double rf, int prec, double *D,
                       int32_t *hubs_out, int32_t *nearest_out, double *dnear_out)
{
    if (n < 1 || (prec != 32 && prec != 64)) return OR_EINVAL;
    int64_t h = n_hubs > 0 ? n_hubs : (int64_t)ceil(sqrt((double)n));
    if (h > n) h = n;
    if (!(rf > 0.0)) rf = 2.0;
    mat_t m = {S, n, ld, dtype};
    graph_t g;
    int rc = build_graph(&m, n, edges, ne, prec, &g);
    if (rc) return rc;
    int32_t *hubs = (int32_t *)malloc(sizeof(int32_t) * (size_t)h);
    double *DH = (double *)malloc(sizeof(double) * (size_t)(h * n));
    int32_t *hn = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *dn = (double *)malloc(sizeof(double) * (size_t)n);
    double *rad = (double *)malloc(sizeof(double) * (size_t)n);
    double *B = (double *)malloc(sizeof(double) * (size_t)(n * n));
    if (!hubs || !DH || !hn || !dn || !rad || !B) { rc = OR_ENOMEM; goto out; }
    rc = oracle_hubs(n, edges, ne, h, hubs);
    if (rc) goto out;
    /* exact SSSP from every hub, then (below) the bounded searches: each
       search is independent, so they run on all host threads */
#pragma omp parallel
    {
        uint8_t *done = (uint8_t *)malloc((size_t)n);
        dent_t *heap = (dent_t *)malloc(sizeof(dent_t) * (size_t)(2 * ne + n + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < h; ++i)
            if (done && heap) dijkstra(&g, hubs[i], prec, -1.0, DH + i * n, done, heap);
        if (!done || !heap) {
#pragma omp atomic write
            rc = OR_ENOMEM;
        }
        free(done); free(heap);
    }
    if (rc) goto out;
    /* nearest hub and radius of every source */
    for (int64_t s = 0; s < n; ++s) {
        int32_t bi = 0;
        for (int64_t i = 1; i < h; ++i)
            if (DH[i * n + s] < DH[bi * n + s]) bi = (int32_t)i;
        hn[s] = bi;
        dn[s] = DH[bi * n + s];
        rad[s] = prec == 32 ? (double)((float)rf * (float)dn[s]) : rf * dn[s];
    }
    /* bounded exact search from every source */
#pragma omp parallel
    {
        uint8_t *done = (uint8_t *)malloc((size_t)n);
        dent_t *heap = (dent_t *)malloc(sizeof(dent_t) * (size_t)(2 * ne + n + 1));
#pragma omp for schedule(dynamic, 64)
        for (int64_t s = 0; s < n; ++s)
            if (done && heap) dijkstra(&g, (int32_t)s, prec, rad[s], B + s * n, done, heap);
        if (!done || !heap) {
#pragma omp atomic write
            rc = OR_ENOMEM;
        }
        free(done); free(heap);
    }
    if (rc) goto out;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s)
        for (int64_t t = 0; t < n; ++t) {
            double est_s, est_t, v;
            if (prec == 32) {
                est_s = (double)((float)dn[s] + (float)DH[(int64_t)hn[s] * n + t]);
                est_t = (double)((float)dn[t] + (float)DH[(int64_t)hn[t] * n + s]);
            } else {
                est_s = dn[s] + DH[(int64_t)hn[s] * n + t];
                est_t = dn[t] + DH[(int64_t)hn[t] * n + s];
            }
            v = est_s < est_t ? est_s : est_t;
            if (B[s * n + t] <= rad[s] && B[s * n + t] < v) v = B[s * n + t];
            if (B[t * n + s] <= rad[t] && B[t * n + s] < v) v = B[t * n + s];
            D[s * n + t] = v;
        }
    if (hubs_out) memcpy(hubs_out, hubs, sizeof(int32_t) * (size_t)h);
    if (nearest_out) memcpy(nearest_out, hn, sizeof(int32_t) * (size_t)n);
    if (dnear_out) memcpy(dnear_out, dn, sizeof(double) * (size_t)n);
out:
    free(hubs); free(DH); free(hn); free(dn); free(rad); free(B);
    graph_free(&g);
    return rc;
}

/* Rows of the approximate APSP (Section 4.3; reading R12) for the listed
 * sources only: row i of D (nsrc x n) equals row src[i] of oracle_apsp_approx
 * with the same arguments, without its n x n work matrix.  The bounded search
 * from every vertex t still runs (its distance to a listed source enters
 * D[s,t] when within t's radius); only those distances are kept. */
int oracle_apsp_approx_rows(const void *S, int64_t n, int64_t ld, int dtype,
                            const int32_t *edges, int64_t ne, int64_t n_hubs, double rf,
                            int prec, const int32_t *src, int64_t nsrc, double *D)
{
    if (n < 1 || nsrc < 0 || (prec != 32 && prec != 64)) return OR_EINVAL;
    for (int64_t i = 0; i < nsrc; ++i)
        if (src[i] < 0 || src[i] >= n) return OR_EINVAL;
    int64_t h = n_hubs > 0 ? n_hubs : (int64_t)ceil(sqrt((double)n));
    if (h > n) h = n;
    if (!(rf > 0.0)) rf = 2.0;
    mat_t m = {S, n, ld, dtype};
    graph_t g;
    int rc = build_graph(&m, n, edges, ne, prec, &g);
    if (rc) return rc;
    int32_t *hubs = (int32_t *)malloc(sizeof(int32_t) * (size_t)h);
    double *DH = (double *)malloc(sizeof(double) * (size_t)(h * n));
    int32_t *hn = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *dn = (double *)malloc(sizeof(double) * (size_t)n);
    double *rad = (double *)malloc(sizeof(double) * (size_t)n);
    double *Bs = (double *)malloc(sizeof(double) * (size_t)(nsrc * n + 1)); /* from s */
    double *Bt = (double *)malloc(sizeof(double) * (size_t)(nsrc * n + 1)); /* from t, at s */
    if (!hubs || !DH || !hn || !dn || !rad || !Bs || !Bt) { rc = OR_ENOMEM; goto out; }
    rc = oracle_hubs(n, edges, ne, h, hubs);
    if (rc) goto out;
#pragma omp parallel
    {
        uint8_t *done = (uint8_t *)malloc((size_t)n);
        dent_t *heap = (dent_t *)malloc(sizeof(dent_t) * (size_t)(2 * ne + n + 1));
        double *row = (double *)malloc(sizeof(double) * (size_t)n);
        int ok = done && heap && row;
        /* exact SSSP from every hub */
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < h; ++i)
            if (ok) dijkstra(&g, hubs[i], prec, -1.0, DH + i * n, done, heap);
        /* nearest hub and radius of every vertex */
#pragma omp for schedule(static)
        for (int64_t s = 0; s < n; ++s) {
            int32_t bi = 0;
            for (int64_t i = 1; i < h; ++i)
                if (DH[i * n + s] < DH[bi * n + s]) bi = (int32_t)i;
            hn[s] = bi;
            dn[s] = DH[bi * n + s];
            rad[s] = prec == 32 ? (double)((float)rf * (float)dn[s]) : rf * dn[s];
        }
        /* bounded searches from the listed sources, and from every vertex t
           with only its distances to the listed sources kept */
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < nsrc; ++i)
            if (ok) dijkstra(&g, src[i], prec, rad[src[i]], Bs + i * n, done, heap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < n; ++t) {
            if (!ok) continue;
            dijkstra(&g, (int32_t)t, prec, rad[t], row, done, heap);
            for (int64_t i = 0; i < nsrc; ++i) Bt[i * n + t] = row[src[i]];
        }
        if (!ok) {
#pragma omp atomic write
            rc = OR_ENOMEM;
        }
        free(done); free(heap); free(row);
    }
    if (rc) goto out;
    for (int64_t i = 0; i < nsrc; ++i) {
        const int64_t s = src[i];
        for (int64_t t = 0; t < n; ++t) {
            double est_s, est_t, v;
            if (prec == 32) {
                est_s = (double)((float)dn[s] + (float)DH[(int64_t)hn[s] * n + t]);
                est_t = (double)((float)dn[t] + (float)DH[(int64_t)hn[t] * n + s]);
            } else {
                est_s = dn[s] + DH[(int64_t)hn[s] * n + t];
                est_t = dn[t] + DH[(int64_t)hn[t] * n + s];
            }
            v = est_s < est_t ? est_s : est_t;
            if (Bs[i * n + t] <= rad[s] && Bs[i * n + t] < v) v = Bs[i * n + t];
            if (Bt[i * n + t] <= rad[t] && Bt[i * n + t] < v) v = Bt[i * n + t];
            D[i * n + t] = v;
        }
    }
out:
    free(hubs); free(DH); free(hn); free(dn); free(rad); free(Bs); free(Bt);
    graph_free(&g);
    return rc;
}

/* ------------------------------------------------------------------ */
/* complete linkage (used by DBHT)                                      */
/* ------------------------------------------------------------------ */

/* Complete linkage of m items whose pairwise distances are dist(i,j) =
 * dm[i*m+j].  Items carry cluster ids ids[i] and "representatives" rep[i]
 * (the smallest leaf id they contain) and sizes sz[i].  At each merge the
 * pair with the smallest distance is taken; ties go to the pair with the
 * smallest (min(rep), max(rep)).  Each merge writes one linkage row
 * (id_lo, id_hi, height, size) starting at row *next_row and creates the
 * cluster id n + row.  On return ids[0] is the id of the final cluster.
 * dm is destroyed. */
static void complete_linkage(int64_t m, double *dm, int64_t *ids, int64_t *rep, int64_t *sz,
                             int64_t n_leaves, double *Z, int64_t *next_row)
{
    uint8_t *alive = (uint8_t *)malloc((size_t)m);
    for (int64_t i = 0; i < m; ++i) alive[i] = 1;
    for (int64_t step = 0; step + 1 < m; ++step) {
        int64_t bi = -1, bj = -1;
        double bd = INFINITY;
        int64_t br0 = 0, br1 = 0;
        for (int64_t i = 0; i < m; ++i) {
            if (!alive[i]) continue;
            for (int64_t j = i + 1; j < m; ++j) {
                if (!alive[j]) continue;
                double d = dm[i * m + j];
                int64_t r0 = rep[i] < rep[j] ? rep[i] : rep[j];
                int64_t r1 = rep[i] < rep[j] ? rep[j] : rep[i];
                if (bi < 0 || d < bd || (d == bd && (r0 < br0 || (r0 == br0 && r1 < br1)))) {
                    bi = i; bj = j; bd = d; br0 = r0; br1 = r1;
                }
            }
        }
        int64_t row = (*next_row)++;
        int64_t a = ids[bi], b = ids[bj];
        Z[4 * row + 0] = (double)(a < b ? a : b);
        Z[4 * row + 1] = (double)(a < b ? b : a);
        Z[4 * row + 2] = bd;
        Z[4 * row + 3] = (double)(sz[bi] + sz[bj]);
        /* merged cluster lives in slot bi */
        for (int64_t k = 0; k < m; ++k) {
            if (!alive[k] || k == bi || k == bj) continue;
            double d1 = dm[bi * m + k], d2 = dm[bj * m + k];
            double d = d1 > d2 ? d1 : d2;
            dm[bi * m + k] = d;
            dm[k * m + bi] = d;
        }
        ids[bi] = n_leaves + row;
        rep[bi] = rep[bi] < rep[bj] ? rep[bi] : rep[bj];
        sz[bi] += sz[bj];
        alive[bj] = 0;
    }
    /* move the surviving cluster to slot 0 */
    for (int64_t i = 0; i < m; ++i)
        if (alive[i]) { ids[0] = ids[i]; rep[0] = rep[i]; sz[0] = sz[i]; break; }
    free(alive);
}

/* Plain complete linkage of n points under the full distance matrix
 * D (n x n, row-major, symmetric part used: dist(i,j) = D[min,max]).
 * Z: (n-1) x 4 linkage in the layout (id_lo, id_hi, height, size). */
int oracle_complete_linkage(const double *D, int64_t n, double *Z)
{
    if (n < 1) return OR_EINVAL;
    double *dm = (double *)malloc(sizeof(double) * (size_t)(n * n));
    int64_t *ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *rep = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *sz = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!dm || !ids || !rep || !sz) { free(dm); free(ids); free(rep); free(sz); return OR_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        ids[i] = i; rep[i] = i; sz[i] = 1;
        for (int64_t j = 0; j < n; ++j) dm[i * n + j] = i < j ? D[i * n + j] : D[j * n + i];
    }
    int64_t row = 0;
    complete_linkage(n, dm, ids, rep, sz, n, Z, &row);
    free(dm); free(ids); free(rep); free(sz);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* DBHT (Section 2, "PMFG, TMFG, and DBHT"; reading R13)                 */
/* ------------------------------------------------------------------ */
/*
 * R13, the reading of the DBHT sketch:
 *  (a) Bubbles: bubble 0 = the initial clique, bubble k = {v_k} + t_k.  The
 *      bubble-tree edge between parent(k) and k crosses triangle t_k.
 *  (b) Direction: removing t_k splits the other vertices into inside(k)
 *      (vertices of the bubbles in the subtree of k, minus t_k) and the
 *      rest.  w_in / w_out = sum of q(S[i,j]) (q as in R2, exact int64)
 *      over TMFG edges (i,j) with i in t_k and j inside / outside.  The
 *      edge points toward the inside (parent -> k) iff w_in > w_out, else
 *      toward the parent.
 *  (c) Converging bubbles: bubbles with no outgoing edge.
 *  (d) Group of a vertex v: the converging bubble c minimising the mean of
 *      D[v,u] over u in c (ties to the smaller bubble id).
 *  (e) Bubble home: a converging bubble belongs to its own group; any other
 *      bubble b to the converging bubble c minimising the mean of D[i,j]
 *      over i in b, j in c (ties to the smaller bubble id).
 *  (f) Bubble of a vertex v: among the bubbles whose home is v's group, the
 *      one minimising the mean of D[v,u] over u in it (ties: smaller id).
 *  (g) Linkage: complete linkage on D among the vertices of each (group,
 *      bubble) cell, then among the cells of each group, then among the
 *      groups; all ties as in complete_linkage above.  Means are taken in
 *      double, summing over u in ascending id order.
 *  Distances D[i,j] are read as D[min(i,j), max(i,j)].
 */

static double dsym(const double *D, int64_t n, int64_t i, int64_t j)
{
    return i <= j ? D[i * n + j] : D[j * n + i];
}

/* Outputs: Z (n-1)x4; optional dir[n-4] (1: parent->k toward inside,
 * 0: k->parent), converging[n-3] flags, group[n] (converging bubble id),
 * bubble_of[n]. */
int oracle_dbht(const void *S, int64_t n, int64_t ld, int dtype, const int32_t *order,
                const int32_t *edges, const int32_t *ins_face, const int32_t *parent,
                const double *D, double *Z, int32_t *dir_out, int32_t *conv_out,
                int32_t *group_out, int32_t *bubble_out)
{
    if (n < 4) return OR_EINVAL;
    mat_t m = {S, n, ld, dtype};
    int64_t nb = n - 3, ne = 3 * n - 6;
    int rc = OR_OK;
    int32_t *bv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(4 * nb)); /* bubble vertices */
    int32_t *dir = (int32_t *)calloc((size_t)nb, sizeof(int32_t));
    int32_t *outdeg = (int32_t *)calloc((size_t)nb, sizeof(int32_t));
    uint8_t *inside = (uint8_t *)malloc((size_t)n);
    uint8_t *insub = (uint8_t *)malloc((size_t)nb);
    int32_t *group = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *home = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    int32_t *bub = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *conv = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    if (!bv || !dir || !outdeg || !inside || !insub || !group || !home || !bub || !conv) {
        rc = OR_ENOMEM;
        goto out;
    }
    /* (a) bubble vertex sets: the clique, then each insertion's vertex and face */
    for (int i = 0; i < 4; ++i) bv[i] = order[i];
    for (int64_t k = 1; k < nb; ++k) {
        bv[4 * k + 0] = order[4 + k - 1];
        for (int j = 0; j < 3; ++j) bv[4 * k + 1 + j] = ins_face[3 * (k - 1) + j];
    }
    /* (b) directions */
    for (int64_t k = 1; k < nb; ++k) {
        /* subtree of k: bubbles created after k descend from k iff the
           parent chain reaches k (parents always have smaller ids) */
        memset(insub, 0, (size_t)nb);
        insub[k] = 1;
        for (int64_t j = k + 1; j < nb; ++j) insub[j] = insub[parent[j]];
        memset(inside, 0, (size_t)n);
        for (int64_t j = k; j < nb; ++j)
            if (insub[j])
                for (int i = 0; i < 4; ++i) inside[bv[4 * j + i]] = 1;
        const int32_t *t = ins_face + 3 * (k - 1);
        for (int i = 0; i < 3; ++i) inside[t[i]] = 0;
        int64_t w_in = 0, w_out = 0;
        for (int64_t e = 0; e < ne; ++e) {
            int32_t a = edges[2 * e], b = edges[2 * e + 1];
            int a_t = (a == t[0] || a == t[1] || a == t[2]);
            int b_t = (b == t[0] || b == t[1] || b == t[2]);
            if (a_t == b_t) continue; /* both in t or neither */
            int32_t j = a_t ? b : a;
            int64_t q = oracle_quantize(sget(&m, a, b));
            if (inside[j]) w_in += q; else w_out += q;
        }
        dir[k] = w_in > w_out ? 1 : 0;
        if (dir[k]) outdeg[parent[k]]++; else outdeg[k]++;
    }
    /* (c) converging bubbles */
    int64_t nc = 0;
    for (int64_t b = 0; b < nb; ++b)
        if (outdeg[b] == 0) conv[nc++] = (int32_t)b;
    /* (d) group of each vertex */
    for (int64_t v = 0; v < n; ++v) {
        int32_t bc = -1;
        double bm = INFINITY;
        for (int64_t c = 0; c < nc; ++c) {
            double s = 0.0;
            for (int i = 0; i < 4; ++i) s += dsym(D, n, v, bv[4 * conv[c] + i]);
            s = s / 4.0;
            if (bc < 0 || s < bm) { bc = conv[c]; bm = s; }
        }
        group[v] = bc;
    }
    /* (e) home of each bubble */
    for (int64_t b = 0; b < nb; ++b) {
        if (outdeg[b] == 0) { home[b] = (int32_t)b; continue; }
        int32_t bc = -1;
        double bm = INFINITY;
        for (int64_t c = 0; c < nc; ++c) {
            double s = 0.0;
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) s += dsym(D, n, bv[4 * b + i], bv[4 * conv[c] + j]);
            s = s / 16.0;
            if (bc < 0 || s < bm) { bc = conv[c]; bm = s; }
        }
        home[b] = bc;
    }
    /* (f) bubble of each vertex */
    for (int64_t v = 0; v < n; ++v) {
        int32_t bb = -1;
        double bm = INFINITY;
        for (int64_t b = 0; b < nb; ++b) {
            if (home[b] != group[v]) continue;
            double s = 0.0;
            for (int i = 0; i < 4; ++i) s += dsym(D, n, v, bv[4 * b + i]);
            s = s / 4.0;
            if (bb < 0 || s < bm) { bb = (int32_t)b; bm = s; }
        }
        bub[v] = bb;
    }
    /* (g) three-level complete linkage */
    {
        int64_t row = 0;
        int64_t *cell_id = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
        int64_t *cell_rep = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
        int64_t *cell_sz = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
        int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        int64_t *ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        int64_t *rep = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        int64_t *sz = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)n); /* local index */
        int64_t *bslot = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
        int64_t *gslot = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
        int64_t *grp_id = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
        int64_t *grp_rep = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
        int64_t *grp_sz = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
        double *dm = (double *)malloc(sizeof(double) * (size_t)(n * n));
        if (!cell_id || !cell_rep || !cell_sz || !members || !ids || !rep || !sz || !slot ||
            !bslot || !gslot || !grp_id || !grp_rep || !grp_sz || !dm) {
            rc = OR_ENOMEM;
        } else {
            /* level 1: the vertices of each (group, bubble) cell */
            for (int64_t b = 0; b < nb; ++b) {
                cell_id[b] = -1;
                int64_t cnt = 0;
                for (int64_t v = 0; v < n; ++v)
                    if (bub[v] == b) members[cnt++] = v;
                if (!cnt) continue;
                for (int64_t i = 0; i < cnt; ++i) {
                    ids[i] = members[i]; rep[i] = members[i]; sz[i] = 1;
                    for (int64_t j = 0; j < cnt; ++j)
                        dm[i * cnt + j] = dsym(D, n, members[i], members[j]);
                }
                complete_linkage(cnt, dm, ids, rep, sz, n, Z, &row);
                cell_id[b] = ids[0]; cell_rep[b] = rep[0]; cell_sz[b] = sz[0];
            }
            /* level 2: the cells of each group; cluster distance = the
               largest D over a pair of member vertices */
            int64_t ngrp = 0;
            for (int64_t c = 0; c < nc; ++c) {
                int64_t cnt = 0;
                for (int64_t b = 0; b < nb; ++b) {
                    bslot[b] = -1;
                    if (cell_id[b] >= 0 && home[b] == conv[c]) {
                        bslot[b] = cnt;
                        ids[cnt] = cell_id[b]; rep[cnt] = cell_rep[b]; sz[cnt] = cell_sz[b];
                        ++cnt;
                    }
                }
                gslot[c] = -1;
                if (!cnt) continue;
                for (int64_t i = 0; i < cnt * cnt; ++i) dm[i] = 0.0;
                for (int64_t u = 0; u < n; ++u) {
                    if (group[u] != conv[c]) continue;
                    for (int64_t w = 0; w < n; ++w) {
                        if (group[w] != conv[c]) continue;
                        int64_t i = bslot[bub[u]], j = bslot[bub[w]];
                        if (i == j) continue;
                        double d = dsym(D, n, u, w);
                        if (d > dm[i * cnt + j]) dm[i * cnt + j] = d;
                    }
                }
                complete_linkage(cnt, dm, ids, rep, sz, n, Z, &row);
                gslot[c] = ngrp;
                grp_id[ngrp] = ids[0]; grp_rep[ngrp] = rep[0]; grp_sz[ngrp] = sz[0];
                ++ngrp;
            }
            /* level 3: the groups */
            for (int64_t v = 0; v < n; ++v) {
                int64_t c;
                for (c = 0; c < nc; ++c)
                    if (conv[c] == group[v]) break;
                slot[v] = gslot[c];
            }
            for (int64_t i = 0; i < ngrp; ++i) {
                ids[i] = grp_id[i]; rep[i] = grp_rep[i]; sz[i] = grp_sz[i];
            }
            for (int64_t i = 0; i < ngrp * ngrp; ++i) dm[i] = 0.0;
            for (int64_t u = 0; u < n; ++u)
                for (int64_t w = 0; w < n; ++w) {
                    int64_t i = slot[u], j = slot[w];
                    if (i == j) continue;
                    double d = dsym(D, n, u, w);
                    if (d > dm[i * ngrp + j]) dm[i * ngrp + j] = d;
                }
            complete_linkage(ngrp, dm, ids, rep, sz, n, Z, &row);
            if (row != n - 1) rc = OR_EINVAL;
        }
        free(cell_id); free(cell_rep); free(cell_sz); free(members); free(ids); free(rep);
        free(sz); free(slot); free(bslot); free(gslot); free(grp_id); free(grp_rep); free(grp_sz);
        free(dm);
    }
    if (dir_out) for (int64_t k = 1; k < nb; ++k) dir_out[k - 1] = dir[k];
    if (conv_out) for (int64_t b = 0; b < nb; ++b) conv_out[b] = outdeg[b] == 0;
    if (group_out) memcpy(group_out, group, sizeof(int32_t) * (size_t)n);
    if (bubble_out) memcpy(bubble_out, bub, sizeof(int32_t) * (size_t)n);
out:
    free(bv); free(dir); free(outdeg); free(inside); free(insub); free(group); free(home);
    free(bub); free(conv);
    return rc;
}

/* ------------------------------------------------------------------ */
/* evaluation (Section 5): dendrogram cut and ARI                        */
/* ------------------------------------------------------------------ */

/* Cut so that k clusters remain: apply the first n-k merges of Z.  Labels
 * are numbered 0..k-1 in the order of each cluster's smallest member. */
int oracle_cut(const double *Z, int64_t n, int64_t k, int32_t *labels)
{
    if (k < 1 || k > n) return OR_EINVAL;
    int64_t *uf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * n));
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * n));
    if (!uf || !lab) { free(uf); free(lab); return OR_ENOMEM; }
    for (int64_t i = 0; i < 2 * n; ++i) uf[i] = i;
    for (int64_t r = 0; r < n - k; ++r) {
        int64_t a = (int64_t)Z[4 * r], b = (int64_t)Z[4 * r + 1];
        uf[a] = n + r;
        uf[b] = n + r;
    }
    for (int64_t i = 0; i < 2 * n; ++i) lab[i] = -1;
    int32_t next = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t r = v;
        while (uf[r] != r) r = uf[r];
        if (lab[r] < 0) lab[r] = next++;
        labels[v] = lab[r];
    }
    free(uf); free(lab);
    return OR_OK;
}

static double choose2(double x) { return x * (x - 1.0) / 2.0; }

/* Adjusted Rand index, written as in Section 5 (Hubert & Arabie). */
double oracle_ari(const int32_t *truth, const int32_t *pred, int64_t n)
{
    int32_t a_max = 0, b_max = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (truth[i] > a_max) a_max = truth[i];
        if (pred[i] > b_max) b_max = pred[i];
    }
    int64_t A = a_max + 1, B = b_max + 1;
    int64_t *nij = (int64_t *)calloc((size_t)(A * B), sizeof(int64_t));
    int64_t *ni = (int64_t *)calloc((size_t)A, sizeof(int64_t));
    int64_t *nj = (int64_t *)calloc((size_t)B, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        nij[truth[i] * B + pred[i]]++;
        ni[truth[i]]++;
        nj[pred[i]]++;
    }
    double sij = 0.0, si = 0.0, sj = 0.0;
    for (int64_t i = 0; i < A * B; ++i) sij += choose2((double)nij[i]);
    for (int64_t i = 0; i < A; ++i) si += choose2((double)ni[i]);
    for (int64_t j = 0; j < B; ++j) sj += choose2((double)nj[j]);
    double expected = si * sj / choose2((double)n);
    double maxidx = 0.5 * (si + sj);
    free(nij); free(ni); free(nj);
    if (maxidx == expected) return 1.0; /* both partitions trivial and identical */
    return (sij - expected) / (maxidx - expected);
}

/* ------------------------------------------------------------------ */
/* Pearson similarity (Section 5, Datasets) in double                    */
/* ------------------------------------------------------------------ */

/* X: n series of length T (row-major, float or double per dtype).
 * S: n x n doubles, rho_ij = sum (x_i - mu_i)(x_j - mu_j) /
 *    sqrt(sum (x_i - mu_i)^2 * sum (x_j - mu_j)^2). */
int oracle_pearson(const void *X, int64_t n, int64_t T, int dtype, double *S)
{
    if (n < 1 || T < 2) return OR_EINVAL;
    double *Xc = (double *)malloc(sizeof(double) * (size_t)(n * T));
    double *nrm = (double *)malloc(sizeof(double) * (size_t)n);
    if (!Xc || !nrm) { free(Xc); free(nrm); return OR_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        double mu = 0.0;
        for (int64_t t = 0; t < T; ++t)
            mu += dtype == OR_F32 ? (double)((const float *)X)[i * T + t] : ((const double *)X)[i * T + t];
        mu /= (double)T;
        double ss = 0.0;
        for (int64_t t = 0; t < T; ++t) {
            double x = dtype == OR_F32 ? (double)((const float *)X)[i * T + t] : ((const double *)X)[i * T + t];
            Xc[i * T + t] = x - mu;
            ss += (x - mu) * (x - mu);
        }
        nrm[i] = sqrt(ss);
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int64_t t = 0; t < T; ++t) s += Xc[i * T + t] * Xc[j * T + t];
            S[i * n + j] = s / (nrm[i] * nrm[j]);
        }
    free(Xc); free(nrm);
    return OR_OK;
}
