/*
 * Seeded synthetic XCSR workloads.
 *
 * This module only draws inputs.  It holds none of the transposition
 * arithmetic: it writes a row-major XCSR matrix (row_ptr, col_idx, cell_ptr,
 * values) and row-block partition boundaries into caller-owned host buffers.
 * The oracle side and the CUDA side both take their inputs from here.
 *
 * Randomness is counter based, so every output is a pure function of
 * (seed, index) and does not depend on the number of threads:
 *   - SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): state advances by the
 *     golden-ratio increment and each output is the mixed state.
 *   - Each row r draws from its own SplitMix64 sequence keyed by
 *     mix(mix(seed, tag), r); each value v draws from the sequence keyed by
 *     mix(seed, tag) at counter v.
 * Distributions:
 *   - Poisson(lambda), small lambda: Knuth's product-of-uniforms method.
 *   - LogNormal(mu, sigma): exp(mu + sigma Z), Z by Box-Muller.
 *   - Geometric(p) on {1, 2, ...}: inversion, 1 + floor(ln U / ln(1 - p)).
 *   - Zipf(s) on {1..N}: rejection-inversion of Hoermann and Derflinger
 *     (ACM TOMACS 6(3), 1996), written from the method's description.
 *   - Uniform integers (row lengths, run lengths): rng_below, a multiply-high
 *     reduction of one 64-bit draw.
 *   - Distinct columns inside a row: rejection of repeats with a small
 *     open-addressing set; each row's columns are then sorted ascending.
 *   - Zipf rank -> column id: a seeded bijection on [0, N) built from a
 *     4-round Feistel network on the enclosing power-of-two domain with
 *     cycle walking (Black and Rogaway, CT-RSA 2002).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYN_OK 0
#define SYN_EINVAL -1
#define SYN_ENOMEM -2

/* row-count distributions */
#define ROW_EXACT 0     /* a = k */
#define ROW_POISSON 1   /* a = lambda */
#define ROW_LOGNORMAL 2 /* a = mu, b = sigma, rounded to nearest */
#define ROW_UNIFORM 3   /* uniform on the integers [a, b] */
/* column distributions (always distinct inside a row) */
#define COL_UNIFORM 0
#define COL_ZIPF 1      /* a = s, perm = 1: seeded bijection rank->column */
/* run-length distributions */
#define LEN_EXACT 0       /* a = k */
#define LEN_ONE_PLUS_POISSON 1 /* 1 + Poisson(a) */
#define LEN_GEOMETRIC 2   /* Geometric(p = 1/a) on {1,2,...}, a = mean */
#define LEN_UNIFORM 3     /* uniform on [len_min, len_max] */
/* payload kinds */
#define PAY_COUNTER 0   /* int64: base + global value index (base from seed) */
#define PAY_BITS 1      /* uniform random bytes */
#define PAY_F32 2       /* fp32 fields uniform in [0, 1) */
#define PAY_ID 3        /* first 8 bytes = global value index, rest random */

typedef struct {
    int64_t n_rows, n_cols;
    int32_t row_dist;
    double row_a, row_b;
    int64_t row_cap;  /* cells per row are clamped to [0, min(row_cap, n_cols)] */
    int32_t col_dist;
    double col_a;
    int32_t col_perm;
    int32_t len_dist;
    double len_a;
    int64_t len_min, len_max; /* runs are clamped to [len_min, len_max] */
    int32_t payload;
    int32_t stride;       /* bytes per value, multiple of 4 */
    int32_t offset_bytes; /* 4 or 8 */
    uint64_t seed;
} syn_spec;

enum { TAG_ROWLEN = 1, TAG_CELLS = 2, TAG_VALS = 3, TAG_PERM = 4, TAG_PART = 5, TAG_BASE = 6,
       TAG_WIDTH = 7, TAG_BYTES = 8 };

static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
#define GOLDEN 0x9e3779b97f4a7c15ULL
static inline uint64_t key2(uint64_t a, uint64_t b) { return sm_mix(a ^ sm_mix(b + GOLDEN)); }

typedef struct { uint64_t s; } rng_t;
static inline rng_t rng_for(uint64_t seed, uint64_t tag, uint64_t idx) {
    rng_t r; r.s = key2(key2(seed, tag), idx); return r;
}
static inline uint64_t rng_next(rng_t *r) { r->s += GOLDEN; return sm_mix(r->s); }
/* uniform in (0, 1]: never 0 so that logs are finite */
static inline double rng_u01(rng_t *r) { return ((rng_next(r) >> 11) + 1) * (1.0 / 9007199254740992.0); }
static inline uint64_t rng_below(rng_t *r, uint64_t n) {
    /* multiply-shift reduction of a 64-bit draw (bias < n / 2^64) */
    return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

static int64_t draw_poisson(rng_t *r, double lambda) {
    double L = exp(-lambda), p = 1.0;
    int64_t k = 0;
    do { k++; p *= rng_u01(r); } while (p > L);
    return k - 1;
}
static double draw_normal(rng_t *r) {
    double u1 = rng_u01(r), u2 = rng_u01(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
static int64_t draw_geometric(rng_t *r, double p) {
    if (p >= 1.0) return 1;
    double u = rng_u01(r);
    double k = floor(log(u) / log1p(-p));
    if (k > 4.0e18) k = 4.0e18;
    return 1 + (int64_t)k;
}

/* ---- Zipf by rejection-inversion ---------------------------------------
 * h(x) = x^-s is the unnormalised mass; H is an antiderivative of h,
 * H(x) = (x^(1-s) - 1) / (1 - s) (log x when s == 1).  Draw u uniformly in
 * [H(N + 1/2), H(3/2) - h(1)], invert, round to k, and accept k when it lies
 * close enough to the inverse or u is above H(k + 1/2) - h(k). */
typedef struct { double s, hx1, hn, sq; int64_t n; } zipf_t;
static double zh(const zipf_t *z, double x) { return exp(-z->s * log(x)); }
static double zH(const zipf_t *z, double x) {
    double lx = log(x), t = (1.0 - z->s) * lx;
    /* (exp(t) - 1) / (1 - s) computed stably */
    if (fabs(t) > 1e-8) return expm1(t) / (1.0 - z->s);
    return lx * (1.0 + 0.5 * t);
}
static double zHinv(const zipf_t *z, double y) {
    double t = y * (1.0 - z->s);
    if (t < -1.0) t = -1.0;
    double l = (fabs(t) > 1e-8) ? log1p(t) / (1.0 - z->s) : y * (1.0 - 0.5 * t);
    return exp(l);
}
static void zipf_init(zipf_t *z, double s, int64_t n) {
    z->s = s; z->n = n;
    z->hx1 = zH(z, 1.5) - 1.0;
    z->hn = zH(z, (double)n + 0.5);
    z->sq = 2.0 - zHinv(z, zH(z, 2.5) - zh(z, 2.0));
}
static int64_t zipf_draw(const zipf_t *z, rng_t *r) {
    for (;;) {
        double u = z->hn + rng_u01(r) * (z->hx1 - z->hn);
        double x = zHinv(z, u);
        int64_t k = (int64_t)(x + 0.5);
        if (k < 1) k = 1;
        if (k > z->n) k = z->n;
        if ((double)k - x <= z->sq || u >= zH(z, (double)k + 0.5) - zh(z, (double)k)) return k;
    }
}

/* ---- seeded bijection on [0, n) ---------------------------------------- */
typedef struct { int bits, lb, rbits; uint64_t keys[4]; int64_t n; } perm_t;
static void perm_init(perm_t *p, uint64_t seed, int64_t n) {
    int bits = 1;
    while (bits < 62 && ((int64_t)1 << bits) < n) bits++;
    if (bits < 2) bits = 2;
    p->bits = bits; p->lb = bits / 2; p->rbits = bits - bits / 2; p->n = n;
    for (int i = 0; i < 4; i++) p->keys[i] = key2(key2(seed, TAG_PERM), (uint64_t)i);
}
static uint64_t perm_once(const perm_t *p, uint64_t x) {
    uint64_t lmask = ((uint64_t)1 << p->lb) - 1, rmask = ((uint64_t)1 << p->rbits) - 1;
    uint64_t L = x >> p->rbits, R = x & rmask; /* L has lb bits, R has rbits bits */
    for (int i = 0; i < 4; i++) {
        /* unbalanced Feistel: alternate which half absorbs the round function */
        if ((i & 1) == 0) L = (L ^ sm_mix(R ^ p->keys[i])) & lmask;
        else R = (R ^ sm_mix(L ^ p->keys[i])) & rmask;
    }
    return (L << p->rbits) | R;
}
static int64_t perm_apply(const perm_t *p, int64_t x) {
    uint64_t y = (uint64_t)x;
    do { y = perm_once(p, y); } while (y >= (uint64_t)p->n);
    return (int64_t)y;
}

/* ---- small open-addressing set for distinct draws in one row ------------ */
typedef struct { int64_t *slot; int64_t cap; } iset_t;
static int iset_reset(iset_t *s, int64_t want) {
    int64_t cap = 16;
    while (cap < 2 * want + 2) cap <<= 1;
    if (cap > s->cap) {
        free(s->slot);
        s->slot = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
        if (!s->slot) { s->cap = 0; return -1; }
        s->cap = cap;
    }
    for (int64_t i = 0; i < cap; i++) s->slot[i] = -1;
    s->cap = cap;
    return 0;
}
static int iset_insert(iset_t *s, int64_t v) { /* 1 if newly inserted */
    uint64_t m = (uint64_t)s->cap - 1, h = sm_mix((uint64_t)v) & m;
    for (;;) {
        if (s->slot[h] == -1) { s->slot[h] = v; return 1; }
        if (s->slot[h] == v) return 0;
        h = (h + 1) & m;
    }
}
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ---- thread pool helper -------------------------------------------------- */
typedef struct { void (*fn)(void *, int64_t, int64_t, int); void *ctx; int64_t n; int nt; int id; } job_t;
static void *job_run(void *a) {
    job_t *j = (job_t *)a;
    int64_t lo = j->n * j->id / j->nt, hi = j->n * (j->id + 1) / j->nt;
    j->fn(j->ctx, lo, hi, j->id);
    return NULL;
}
static void parallel_for(int nt, int64_t n, void (*fn)(void *, int64_t, int64_t, int), void *ctx) {
    if (nt < 1) nt = 1;
    if (nt > 256) nt = 256;
    if (n < 4096 || nt == 1) { fn(ctx, 0, n, 0); return; }
    pthread_t th[256];
    job_t jobs[256];
    for (int i = 0; i < nt; i++) {
        jobs[i].fn = fn; jobs[i].ctx = ctx; jobs[i].n = n; jobs[i].nt = nt; jobs[i].id = i;
        if (pthread_create(&th[i], NULL, job_run, &jobs[i]) != 0) { job_run(&jobs[i]); th[i] = 0; }
    }
    for (int i = 0; i < nt; i++) if (th[i]) pthread_join(th[i], NULL);
}

static inline int64_t ld_off(const void *p, int o, int64_t i) {
    return o == 4 ? (int64_t)((const int32_t *)p)[i] : ((const int64_t *)p)[i];
}
static inline void st_off(void *p, int o, int64_t i, int64_t v) {
    if (o == 4) ((int32_t *)p)[i] = (int32_t)v; else ((int64_t *)p)[i] = v;
}

static int spec_ok(const syn_spec *s) {
    if (s->n_rows < 0 || s->n_cols < 0) return 0;
    if (s->offset_bytes != 4 && s->offset_bytes != 8) return 0;
    if (s->stride <= 0 || (s->stride % 4) != 0) return 0;
    if ((s->payload == PAY_COUNTER || s->payload == PAY_ID) && s->stride < 8) return 0;
    if (s->n_cols > 2147483647LL) return 0;
    return 1;
}

static int64_t row_len_of(const syn_spec *s, int64_t r) {
    rng_t g = rng_for(s->seed, TAG_ROWLEN, (uint64_t)r);
    int64_t n;
    switch (s->row_dist) {
    case ROW_POISSON: n = draw_poisson(&g, s->row_a); break;
    case ROW_LOGNORMAL: {
        double x = exp(s->row_a + s->row_b * draw_normal(&g));
        n = (x > 4.0e18) ? (int64_t)4e18 : (int64_t)floor(x + 0.5);
        break;
    }
    case ROW_UNIFORM: {
        const int64_t lo = (int64_t)s->row_a, hi = (int64_t)s->row_b;
        n = hi > lo ? lo + (int64_t)rng_below(&g, (uint64_t)(hi - lo + 1)) : lo;
        break;
    }
    default: n = (int64_t)s->row_a; break;
    }
    int64_t cap = s->row_cap > 0 ? s->row_cap : s->n_cols;
    if (cap > s->n_cols) cap = s->n_cols;
    if (n > cap) n = cap;
    if (n < 0) n = 0;
    return n;
}

/* pass 1: per-row cell counts into row_ptr[r + 1] (row_ptr[0] = 0); returns C */
typedef struct { const syn_spec *s; void *row_ptr; int64_t *part; } rl_ctx;
static void rl_body(void *c, int64_t lo, int64_t hi, int id) {
    rl_ctx *x = (rl_ctx *)c;
    int64_t sum = 0;
    for (int64_t r = lo; r < hi; r++) {
        int64_t n = row_len_of(x->s, r);
        st_off(x->row_ptr, x->s->offset_bytes, r + 1, n);
        sum += n;
    }
    x->part[id] = sum;
}
typedef struct { const syn_spec *s; void *arr; int o; int64_t *base; } ps_ctx;
static void ps_body(void *c, int64_t lo, int64_t hi, int id) {
    ps_ctx *x = (ps_ctx *)c;
    int64_t acc = x->base[id];
    for (int64_t i = lo; i < hi; i++) {
        acc += ld_off(x->arr, x->o, i + 1);
        st_off(x->arr, x->o, i + 1, acc);
    }
}
/* in-place inclusive prefix over arr[1..n], arr[0] = 0, given per-chunk sums */
static int prefix_inplace(void *arr, int o, int64_t n, int nt, int64_t *part) {
    if (nt > 256) nt = 256;
    if (nt < 1) nt = 1;
    int eff = (n < 4096 || nt == 1) ? 1 : nt;
    int64_t base[256];
    int64_t acc = 0;
    for (int i = 0; i < eff; i++) { base[i] = acc; acc += part[i]; }
    st_off(arr, o, 0, 0);
    ps_ctx x = { NULL, arr, o, base };
    parallel_for(eff, n, ps_body, &x);
    return 0;
}

int64_t syn_row_ptr(const syn_spec *s, void *row_ptr, int nthreads) {
    if (!spec_ok(s)) return SYN_EINVAL;
    int64_t part[256] = {0};
    if (nthreads > 256) nthreads = 256;
    if (nthreads < 1) nthreads = 1;
    rl_ctx x = { s, row_ptr, part };
    int eff = (s->n_rows < 4096 || nthreads == 1) ? 1 : nthreads;
    parallel_for(eff, s->n_rows, rl_body, &x);
    int64_t total = 0;
    for (int i = 0; i < eff; i++) total += part[i];
    if (s->offset_bytes == 4 && total > 2147483647LL) return SYN_EINVAL;
    prefix_inplace(row_ptr, s->offset_bytes, s->n_rows, eff, part);
    return total;
}

/* pass 2: columns (ascending, distinct) and run lengths per row.  Lengths go
 * to cell_ptr[k + 1]; a prefix pass turns them into offsets.  Returns V. */
typedef struct { const syn_spec *s; const void *row_ptr; int32_t *col; void *cell_ptr; int64_t *part; int err; zipf_t zf; perm_t pm; } cl_ctx;
static void cl_body(void *c, int64_t lo, int64_t hi, int id) {
    cl_ctx *x = (cl_ctx *)c;
    const syn_spec *s = x->s;
    int o = s->offset_bytes;
    iset_t set = { NULL, 0 };
    int64_t vsum = 0;
    for (int64_t r = lo; r < hi; r++) {
        int64_t k0 = ld_off(x->row_ptr, o, r), k1 = ld_off(x->row_ptr, o, r + 1), n = k1 - k0;
        rng_t g = rng_for(s->seed, TAG_CELLS, (uint64_t)r);
        if (n > 0) {
            if (iset_reset(&set, n) != 0) { x->err = 1; break; }
            int64_t got = 0;
            while (got < n) {
                int64_t c;
                if (s->col_dist == COL_ZIPF) {
                    int64_t rank = zipf_draw(&x->zf, &g) - 1;
                    c = s->col_perm ? perm_apply(&x->pm, rank) : rank;
                } else {
                    c = (int64_t)rng_below(&g, (uint64_t)s->n_cols);
                }
                if (iset_insert(&set, c)) x->col[k0 + got++] = (int32_t)c;
            }
            qsort(x->col + k0, (size_t)n, sizeof(int32_t), cmp_i32);
        }
        for (int64_t k = k0; k < k1; k++) {
            int64_t len;
            switch (s->len_dist) {
            case LEN_ONE_PLUS_POISSON: len = 1 + draw_poisson(&g, s->len_a); break;
            case LEN_GEOMETRIC: len = draw_geometric(&g, 1.0 / s->len_a); break;
            case LEN_UNIFORM: len = s->len_min + (int64_t)rng_below(&g, (uint64_t)(s->len_max - s->len_min + 1)); break;
            default: len = (int64_t)s->len_a; break;
            }
            if (len < s->len_min) len = s->len_min;
            if (s->len_max >= 0 && len > s->len_max) len = s->len_max;
            st_off(x->cell_ptr, o, k + 1, len);
            vsum += len;
        }
    }
    free(set.slot);
    x->part[id] = vsum;
}
typedef struct { void *cell_ptr; int o; int64_t n; int64_t *part; } cs_ctx;
static void cs_body(void *c, int64_t lo, int64_t hi, int id) {
    cs_ctx *x = (cs_ctx *)c;
    int64_t sum = 0;
    for (int64_t i = lo; i < hi; i++) sum += ld_off(x->cell_ptr, x->o, i + 1);
    x->part[id] = sum;
}

int64_t syn_cells(const syn_spec *s, const void *row_ptr, int32_t *col_idx, void *cell_ptr, int nthreads) {
    if (!spec_ok(s)) return SYN_EINVAL;
    if (nthreads > 256) nthreads = 256;
    if (nthreads < 1) nthreads = 1;
    int o = s->offset_bytes;
    int64_t C = ld_off(row_ptr, o, s->n_rows);
    int64_t part[256] = {0};
    cl_ctx x;
    memset(&x, 0, sizeof(x));
    x.s = s; x.row_ptr = row_ptr; x.col = col_idx; x.cell_ptr = cell_ptr; x.part = part;
    if (s->col_dist == COL_ZIPF) zipf_init(&x.zf, s->col_a, s->n_cols);
    perm_init(&x.pm, s->seed, s->n_cols > 1 ? s->n_cols : 2);
    int eff = (s->n_rows < 4096 || nthreads == 1) ? 1 : nthreads;
    parallel_for(eff, s->n_rows, cl_body, &x);
    if (x.err) return SYN_ENOMEM;
    /* re-chunk the lengths by cell for the prefix pass */
    int64_t cpart[256] = {0};
    cs_ctx y = { cell_ptr, o, C, cpart };
    int effc = (C < 4096 || nthreads == 1) ? 1 : nthreads;
    parallel_for(effc, C, cs_body, &y);
    int64_t V = 0;
    for (int i = 0; i < effc; i++) V += cpart[i];
    if (o == 4 && V > 2147483647LL) return SYN_EINVAL;
    prefix_inplace(cell_ptr, o, C, effc, cpart);
    return V;
}

/* pass 3: payload bytes for values [0, V) */
typedef struct { const syn_spec *s; uint8_t *vals; uint64_t key; int64_t base; } pv_ctx;
static void pv_body(void *c, int64_t lo, int64_t hi, int id) {
    (void)id;
    pv_ctx *x = (pv_ctx *)c;
    const syn_spec *s = x->s;
    int st = s->stride;
    for (int64_t v = lo; v < hi; v++) {
        uint8_t *p = x->vals + (size_t)v * (size_t)st;
        int w0 = 0;
        if (s->payload == PAY_COUNTER) { int64_t id8 = x->base + v; memcpy(p, &id8, 8); w0 = 8; }
        else if (s->payload == PAY_ID) { int64_t id8 = v; memcpy(p, &id8, 8); w0 = 8; }
        int nw = (st + 7) / 8;
        for (int w = w0 / 8; w < nw; w++) {
            uint64_t z = sm_mix(x->key + ((uint64_t)v * (uint64_t)nw + (uint64_t)w + 1) * GOLDEN);
            int take = st - 8 * w < 8 ? st - 8 * w : 8;
            if (s->payload == PAY_F32) {
                uint32_t f[2];
                float a = (float)((z >> 40) * (1.0 / 16777216.0));
                float b = (float)(((z >> 8) & 0xFFFFFFu) * (1.0 / 16777216.0));
                memcpy(&f[0], &a, 4); memcpy(&f[1], &b, 4);
                memcpy(p + 8 * w, f, (size_t)take);
            } else {
                memcpy(p + 8 * w, &z, (size_t)take);
            }
        }
    }
}
int syn_values(const syn_spec *s, int64_t n_values, void *values, int nthreads) {
    if (!spec_ok(s) || n_values < 0) return SYN_EINVAL;
    pv_ctx x = { s, (uint8_t *)values, key2(s->seed, TAG_VALS),
                 (int64_t)(key2(s->seed, TAG_BASE) & 0xFFFFFFFFULL) << 20 };
    parallel_for(nthreads, n_values, pv_body, &x);
    return SYN_OK;
}

/* row-block partition boundaries off[0..P]: kind 0 = equal blocks
 * (off_d = floor(d R / P)); kind 1 = off_d = round(R W_d / W_P) with W the
 * cumulative sum of LogNormal(0, sigma) weights drawn from the seed. */
int syn_partitions(int kind, int64_t n_parts, int64_t n_rows, double sigma, uint64_t seed, int64_t *off) {
    if (n_parts < 1 || n_rows < 0) return SYN_EINVAL;
    off[0] = 0;
    if (kind == 0) {
        for (int64_t d = 1; d <= n_parts; d++) off[d] = (int64_t)(((__int128)d * n_rows) / n_parts);
        return SYN_OK;
    }
    double *w = (double *)malloc((size_t)(n_parts + 1) * sizeof(double));
    if (!w) return SYN_ENOMEM;
    w[0] = 0.0;
    for (int64_t d = 0; d < n_parts; d++) {
        rng_t g = rng_for(seed, TAG_PART, (uint64_t)d);
        w[d + 1] = w[d] + exp(sigma * draw_normal(&g));
    }
    for (int64_t d = 1; d <= n_parts; d++) {
        double x = (double)n_rows * (w[d] / w[n_parts]);
        int64_t b = (int64_t)floor(x + 0.5);
        if (b < off[d - 1]) b = off[d - 1];
        if (b > n_rows) b = n_rows;
        off[d] = b;
    }
    off[n_parts] = n_rows;
    free(w);
    return SYN_OK;
}

/* helpers for batched workloads: matrix m's row count, log-uniform in [lo, hi] */
int64_t syn_loguniform(uint64_t seed, uint64_t tag, uint64_t idx, int64_t lo, int64_t hi) {
    rng_t g = rng_for(seed, 100 + tag, idx);
    double u = rng_u01(&g);
    double x = exp(log((double)lo) + u * (log((double)hi) - log((double)lo)));
    int64_t n = (int64_t)floor(x + 0.5);
    if (n < lo) n = lo;
    if (n > hi) n = hi;
    return n;
}
double syn_uniform01(uint64_t seed, uint64_t tag, uint64_t idx) {
    rng_t g = rng_for(seed, 200 + tag, idx);
    return rng_u01(&g);
}
uint64_t syn_key(uint64_t seed, uint64_t tag, uint64_t idx) { return key2(key2(seed, tag), idx); }
int64_t syn_perm(uint64_t seed, int64_t n, int64_t x) {
    perm_t p; perm_init(&p, seed, n > 1 ? n : 2); return perm_apply(&p, x);
}
int64_t syn_zipf_sample(double s, int64_t n, uint64_t seed, int64_t count, int64_t *out) {
    zipf_t z; zipf_init(&z, s, n);
    rng_t g = rng_for(seed, 300, 0);
    for (int64_t i = 0; i < count; i++) out[i] = zipf_draw(&z, &g);
    return count;
}

/* ---- variable-width values ------------------------------------------------
 * Each value v gets a byte width drawn uniformly from sizes[0 .. n_sizes)
 * (one SplitMix64 draw at counter v of the sequence keyed by (seed,
 * TAG_WIDTH)); val_off[0..V] is the prefix of those widths (the input's own
 * byte offsets).  Returns the total bytes val_off[V], or < 0 on bad args. */
typedef struct { uint64_t key; const int32_t *sizes; int n; int64_t *off; int64_t *part; } vw_ctx;
static void vw_body(void *c, int64_t lo, int64_t hi, int id) {
    vw_ctx *x = (vw_ctx *)c;
    int64_t sum = 0;
    for (int64_t v = lo; v < hi; v++) {
        uint64_t z = sm_mix(x->key + ((uint64_t)v + 1) * GOLDEN);
        int64_t w = x->sizes[(uint64_t)(((unsigned __int128)z * (uint64_t)x->n) >> 64)];
        x->off[v + 1] = w;
        sum += w;
    }
    x->part[id] = sum;
}
int64_t syn_widths(uint64_t seed, int64_t n_values, const int32_t *sizes, int n_sizes,
                   int64_t *val_off, int nthreads) {
    if (n_values < 0 || n_sizes < 1 || !sizes || !val_off) return SYN_EINVAL;
    for (int i = 0; i < n_sizes; i++) if (sizes[i] < 0) return SYN_EINVAL;
    if (nthreads > 256) nthreads = 256;
    if (nthreads < 1) nthreads = 1;
    int64_t part[256] = {0};
    vw_ctx x = { key2(seed, TAG_WIDTH), sizes, n_sizes, val_off, part };
    int eff = (n_values < 4096 || nthreads == 1) ? 1 : nthreads;
    parallel_for(eff, n_values, vw_body, &x);
    prefix_inplace(val_off, 8, n_values, eff, part);
    return val_off[n_values];
}

/* nbytes uniform random bytes (8-byte words at counters of (seed, TAG_BYTES)) */
typedef struct { uint64_t key; uint8_t *out; int64_t n; } vb_ctx;
static void vb_body(void *c, int64_t lo, int64_t hi, int id) {
    (void)id;
    vb_ctx *x = (vb_ctx *)c;
    for (int64_t w = lo; w < hi; w++) {
        uint64_t z = sm_mix(x->key + ((uint64_t)w + 1) * GOLDEN);
        int64_t at = w * 8, take = x->n - at < 8 ? x->n - at : 8;
        memcpy(x->out + at, &z, (size_t)take);
    }
}
int syn_bytes(uint64_t seed, int64_t nbytes, uint8_t *out, int nthreads) {
    if (nbytes < 0 || (nbytes > 0 && !out)) return SYN_EINVAL;
    vb_ctx x = { key2(seed, TAG_BYTES), out, nbytes };
    parallel_for(nthreads, (nbytes + 7) / 8, vb_body, &x);
    return SYN_OK;
}
