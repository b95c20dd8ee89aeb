/*
 * pt_oracle.c -- plain, slow CPU oracle for predicate transfer.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no source with the CUDA library: the
 * structs below are declared here independently of the public header.
 *
 * What it computes (Yang, Zhao, Yu, Koutris, "Predicate Transfer", CIDR'24):
 *   - filter transformation (Section 3.2, "Filter Transformation", Fig. 2):
 *     a table is scanned once; rows that pass the local predicate and every
 *     incoming filter survive, and their outgoing join keys are inserted
 *     into one fresh outgoing filter per outgoing edge;
 *   - the predicate transfer graph (Section 3.2, "Predicate Transfer
 *     Graph"): every join edge points from the smaller table to the bigger;
 *   - the schedule (Section 3.2, "Transfer Schedule", Fig. 3): a forward
 *     pass in topological order, then a backward pass over the reversed
 *     edges whose input is the forward survivors;
 *   - one-direction edges (Section 3.4, outer joins): an edge flagged
 *     O_EDGE_ONE_WAY transfers only from t0 to t1, so only in the pass that
 *     orients it that way; in the other pass no filter is built on it;
 *   - "Filter Type" (Section 3.2): with precise filters (exact key sets) a
 *     transfer is a semi-join; mode exact=1 runs that schedule;
 *   - the Bloom join (Section 2.1, and the BloomJoin baseline of Section 4),
 *     a one-hop transfer in one direction: each edge's filter holds the keys
 *     of its building table's selected rows only and is probed once
 *     (o_one_hop).
 *
 * The paper fixes no hash, filter layout, filter size or number of bits.
 * This library fixes them as follows (the same definitions, written
 * separately, are what the CUDA path implements):
 *   key:    int32 is sign-extended to 64 bits, int64 taken as is (u64).
 *   hash:   H(x) = mix(x ^ seed + G), H(a, b) = mix(H(a) ^ b), with G and
 *           mix() the SplitMix64 increment and output function (Steele,
 *           Lea, Flood, OOPSLA 2014).
 *   filter: nblocks blocks of B bits (B = 256 or 512) stored as uint32
 *           words, block j = words [j*B/32, (j+1)*B/32), bit t of a block
 *           = bit (t & 31) of its word t >> 5.
 *   bits:   block j = ((h >> 32) * nblocks) >> 32; with lo = low 32 bits
 *           of h, h1 = lo mod B, h2 = (lo >> 16) | 1, bit i = (h1 + i*h2)
 *           mod B for i < k (Kirsch-Mitzenmacher double hashing, 2006).
 *   size:   nblocks = max(1, ceil(min(c, n_probe) * bits_per_key / B)),
 *           c = the building visit's survivor count, n_probe = rows of the
 *           table on the other end of the edge.
 *   order:  tables are ranked by (rows, table id); the forward pass visits
 *           them in ascending rank, the backward pass in descending rank.
 *   probe:  incoming filters are probed in ascending level of the building
 *           visit (its longest path from a source of the pass's DAG, so
 *           filters that are finished earlier come first), then ascending
 *           c_b / n_b (survivors of the building visit over its table's
 *           rows, the LIP-style ordering of Section 3.2), then edge id
 *           (probe_order 0); probe_order 1 leaves out the level, 2 is edge
 *           id alone.  The order never changes a result, only how many key
 *           sectors are read.
 *
 * Threads: built plainly (liboracle.so) every loop runs on one thread.  The
 * same source built with -fopenmp (liboracle_omp.so, timing only) splits
 * the per-row loops across threads; every row is still handled by the same
 * statements, the survivor words are formed per word, and filter words are
 * OR-ed atomically, so both builds give identical results.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n_rows;
    int32_t n_cols;
    const void* const* cols;   /* n_cols column base pointers */
    const int32_t* dtypes;     /* 0 = int32, 1 = int64 */
    const uint32_t* sel;       /* selection bitmap, NULL = every row */
} o_table;

typedef struct {
    int32_t t0, ncols, c0[2], t1, c1[2];
    uint32_t flags;  /* bit 0: filters flow only from t0 to t1 (Section 3.4: the edge of a
                        left outer join, t0 the preserved side) */
} o_edge;

#define O_EDGE_ONE_WAY 1u

/* Is edge i active in pass p?  A pass sends each edge's filter from its
 * builder (src in the forward pass, dst in the backward pass) to the other
 * end; a one-way edge only transfers when that builder is its t0, so it is
 * active in exactly one of the two passes (Section 3.4). */
static int o_active(const o_edge* e, const int32_t* src, const int32_t* dst, int32_t p, int32_t i) {
    if (!(e[i].flags & O_EDGE_ONE_WAY)) return 1;
    return (p == 0 ? src[i] : dst[i]) == e[i].t0;
}

typedef struct {
    int32_t bits_per_key, k, block_bits;
    int32_t probe_order;  /* 0: builder level, LIP, edge id; 1: LIP, edge id; 2: edge id */
    uint64_t seed;
} o_cfg;

#define O_SPLITMIX_GAMMA 0x9E3779B97F4A7C15ULL

/* ---- hash ------------------------------------------------------------- */

static uint64_t o_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t o_key(const void* col, int32_t dtype, int64_t row) {
    if (dtype == 0) {
        int64_t v = ((const int32_t*)col)[row]; /* sign extension */
        return (uint64_t)v;
    }
    return (uint64_t)((const int64_t*)col)[row];
}

uint64_t o_hash1(uint64_t x, uint64_t seed) { return o_mix((x ^ seed) + O_SPLITMIX_GAMMA); }

uint64_t o_hash2(uint64_t a, uint64_t b, uint64_t seed) { return o_mix(o_hash1(a, seed) ^ b); }

/* ---- blocked Bloom filter -------------------------------------------- */

int64_t o_nblocks(int64_t c, int64_t n_probe, int32_t bits_per_key, int32_t block_bits) {
    int64_t n_est = c < n_probe ? c : n_probe;
    int64_t nb = (n_est * bits_per_key + block_bits - 1) / block_bits;
    return nb < 1 ? 1 : nb;
}

int64_t o_block_of(uint64_t h, int64_t nblocks) {
    return (int64_t)(((h >> 32) * (uint64_t)nblocks) >> 32);
}

void o_bits_of(uint64_t h, int32_t block_bits, int32_t k, int32_t* pos) {
    uint32_t lo = (uint32_t)h;
    uint32_t h1 = lo & (uint32_t)(block_bits - 1);
    uint32_t h2 = (lo >> 16) | 1u;
    for (int32_t i = 0; i < k; i++) pos[i] = (int32_t)((h1 + (uint32_t)i * h2) & (uint32_t)(block_bits - 1));
}

void o_filter_insert(uint32_t* words, int64_t nblocks, int32_t block_bits, int32_t k, uint64_t h) {
    int32_t pos[64];
    int64_t base = o_block_of(h, nblocks) * (block_bits / 32);
    o_bits_of(h, block_bits, k, pos);
    for (int32_t i = 0; i < k; i++) {
#pragma omp atomic update
        words[base + (pos[i] >> 5)] |= 1u << (pos[i] & 31);
    }
}

int o_filter_probe(const uint32_t* words, int64_t nblocks, int32_t block_bits, int32_t k, uint64_t h) {
    int32_t pos[64];
    int64_t base = o_block_of(h, nblocks) * (block_bits / 32);
    o_bits_of(h, block_bits, k, pos);
    for (int32_t i = 0; i < k; i++)
        if (!((words[base + (pos[i] >> 5)] >> (pos[i] & 31)) & 1u)) return 0;
    return 1;
}

/* threads the per-row loops use (the OpenMP build; 1 in the plain build) */
int o_set_threads(int32_t n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---- predicate transfer graph and order (Section 3.2) ---------------- */

static int o_rank_less(const int64_t* n_rows, int32_t a, int32_t b) {
    if (n_rows[a] != n_rows[b]) return n_rows[a] < n_rows[b];
    return a < b;
}

/* src[e]/dst[e]: forward orientation of edge e (smaller table -> bigger).
 * order[]: tables in ascending rank, a topological order of that DAG.    */
int o_orient(int32_t n_tables, const int64_t* n_rows, int32_t n_edges, const o_edge* e,
             int32_t* src, int32_t* dst, int32_t* order) {
    for (int32_t i = 0; i < n_edges; i++) {
        if (o_rank_less(n_rows, e[i].t0, e[i].t1)) { src[i] = e[i].t0; dst[i] = e[i].t1; }
        else { src[i] = e[i].t1; dst[i] = e[i].t0; }
    }
    for (int32_t i = 0; i < n_tables; i++) order[i] = i;
    for (int32_t i = 1; i < n_tables; i++) {      /* insertion sort by rank */
        int32_t x = order[i], j = i - 1;
        while (j >= 0 && o_rank_less(n_rows, x, order[j])) { order[j + 1] = order[j]; j--; }
        order[j + 1] = x;
    }
    return 0;
}

/* ---- exact key sets (precise filters, Section 3.2 "Filter Type") ----- */

typedef struct { uint64_t a, b; } o_pair;

static int o_pair_cmp(const void* x, const void* y) {
    const o_pair* p = (const o_pair*)x;
    const o_pair* q = (const o_pair*)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

/* ---- one visit's key on one side of an edge -------------------------- */

static void o_side(const o_edge* e, int32_t table, const int32_t** cols) {
    *cols = (e->t0 == table) ? e->c0 : e->c1;
}

static o_pair o_edge_key(const o_table* t, const o_edge* e, int32_t table, int64_t row) {
    const int32_t* c;
    o_pair p;
    o_side(e, table, &c);
    p.a = o_key(t->cols[c[0]], t->dtypes[c[0]], row);
    p.b = e->ncols == 2 ? o_key(t->cols[c[1]], t->dtypes[c[1]], row) : 0;
    return p;
}

static uint64_t o_edge_hash(const o_table* t, const o_edge* e, int32_t table, int64_t row, uint64_t seed) {
    o_pair p = o_edge_key(t, e, table, row);
    return e->ncols == 2 ? o_hash2(p.a, p.b, seed) : o_hash1(p.a, seed);
}

static int o_bit(const uint32_t* bm, int64_t r) { return (int)((bm[r >> 5] >> (r & 31)) & 1u); }

/* number of 32-byte sectors of a column of width w bytes that hold a row
 * whose flag is set (row r lives in sector (r * w) / 32)                 */
static int64_t o_sectors(const unsigned char* flag, int64_t n, int32_t w) {
    int64_t per = 32 / w, cnt = 0;
#pragma omp parallel for schedule(static) reduction(+ : cnt)
    for (int64_t s = 0; s < (n + per - 1) / per; s++) {
        int any = 0;
        for (int64_t r = s * per; r < (s + 1) * per && r < n; r++) any |= flag[r];
        cnt += any;
    }
    return cnt;
}

/* filter configuration and edges in range */
static int o_valid(int32_t n_tables, int32_t n_edges, const o_edge* e, const o_cfg* cfg) {
    int32_t i;
    if (cfg->block_bits != 256 && cfg->block_bits != 512) return 0;
    if (cfg->k < 1 || cfg->k > 16 || cfg->bits_per_key < 1) return 0;
    if (cfg->probe_order < 0 || cfg->probe_order > 2) return 0;
    for (i = 0; i < n_edges; i++) {
        if (e[i].ncols < 1 || e[i].ncols > 2 || e[i].t0 == e[i].t1) return 0;
        if (e[i].flags & ~O_EDGE_ONE_WAY) return 0;
        if (e[i].t0 < 0 || e[i].t0 >= n_tables || e[i].t1 < 0 || e[i].t1 >= n_tables) return 0;
    }
    return 1;
}

/*
 * o_transfer: the full forward + backward predicate transfer.
 *
 * surv[p*n_tables + v]  (caller-owned, ceil(n_v/32) words): survivors of
 *                       table v after pass p (0 = forward, 1 = backward).
 * count[p*n_tables + v]: popcount of that bitmap.
 * filt[p*n_edges + e]   (Bloom mode; caller-owned, at least
 *                       o_nblocks(min(n_t0, n_t1), ...) * B/32 words):
 *                       the filter built on edge e in pass p.
 * nblocks[p*n_edges+e]: its size in blocks (0 in exact mode, and for a
 *                       one-way edge in the pass it is not active in).
 * sectors[(p*n_tables + v)*2 + {0,1}] (nullable): key-column sectors read
 *                       by the probes (each probed column, sectors with a
 *                       row still alive when its edge is probed) and by the
 *                       builds (each distinct build column, sectors with a
 *                       survivor).
 * Returns 0, or -1 on invalid input.
 */
int o_transfer(int32_t n_tables, const o_table* t, int32_t n_edges, const o_edge* e,
               const o_cfg* cfg, int32_t exact, uint32_t* const* surv, int64_t* count,
               uint32_t* const* filt, int64_t* nblocks, int64_t* sectors) {
    int32_t B = cfg->block_bits, K = cfg->k, wpb = cfg->block_bits / 32;
    int32_t v, p, i, j;

    if (!o_valid(n_tables, n_edges, e, cfg)) return -1;

    int64_t* n_rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_tables > 0 ? n_tables : 1));
    int32_t* src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_edges + 1));
    int32_t* dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_edges + 1));
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_tables + 1));
    int32_t* ine = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_edges + 1));
    o_pair** set = (o_pair**)calloc((size_t)(2 * n_edges + 1), sizeof(o_pair*));
    int64_t* set_n = (int64_t*)calloc((size_t)(2 * n_edges + 1), sizeof(int64_t));
    int32_t* lvl = (int32_t*)calloc((size_t)(2 * n_tables + 1), sizeof(int32_t));

    for (v = 0; v < n_tables; v++) n_rows[v] = t[v].n_rows;
    o_orient(n_tables, n_rows, n_edges, e, src, dst, order);

    for (p = 0; p < 2; p++) {
        for (int32_t oi = 0; oi < n_tables; oi++) {
            /* forward: ascending rank; backward: reversed edges, descending rank */
            v = p == 0 ? order[oi] : order[n_tables - 1 - oi];
            int64_t n = n_rows[v];
            const uint32_t* in = p == 0 ? t[v].sel : surv[v];  /* backward starts from forward survivors */
            uint32_t* out = surv[p * n_tables + v];
            unsigned char* alive = (unsigned char*)malloc((size_t)(n > 0 ? n : 1));
            int64_t c = 0, probe_sec = 0, build_sec = 0;

#pragma omp parallel for schedule(static)
            for (int64_t r = 0; r < n; r++) alive[r] = in ? (unsigned char)o_bit(in, r) : 1;

            /* incoming edges of v in this pass; v's level is one more than
               its highest builder's (builders are visited before v) */
            int32_t n_in = 0, lv = 0;
            for (i = 0; i < n_edges; i++) {
                int32_t into = p == 0 ? dst[i] : src[i];
                if (into == v && o_active(e, src, dst, p, i)) {
                    int32_t b = p == 0 ? src[i] : dst[i];
                    ine[n_in++] = i;
                    if (lvl[p * n_tables + b] + 1 > lv) lv = lvl[p * n_tables + b] + 1;
                }
            }
            lvl[p * n_tables + v] = lv;
            /* probe order: builder level (order 0 only), then LIP ratio (orders
               0 and 1), then edge id */
            for (i = 1; i < n_in; i++) {
                int32_t x = ine[i];
                j = i - 1;
                while (j >= 0) {
                    int32_t y = ine[j];
                    int32_t bx = p == 0 ? src[x] : dst[x], by = p == 0 ? src[y] : dst[y];
                    int32_t lx = cfg->probe_order == 0 ? lvl[p * n_tables + bx] : 0;
                    int32_t ly = cfg->probe_order == 0 ? lvl[p * n_tables + by] : 0;
                    uint64_t lhs = cfg->probe_order == 2 ? 0 : (uint64_t)count[p * n_tables + bx] * (uint64_t)n_rows[by];
                    uint64_t rhs = cfg->probe_order == 2 ? 0 : (uint64_t)count[p * n_tables + by] * (uint64_t)n_rows[bx];
                    if (lx < ly || (lx == ly && (lhs < rhs || (lhs == rhs && x < y)))) { ine[j + 1] = ine[j]; j--; }
                    else break;
                }
                ine[j + 1] = x;
            }

            /* probe: a row survives iff it is in the input and every incoming filter accepts its key */
            for (i = 0; i < n_in; i++) {
                const o_edge* ed = &e[ine[i]];
                const int32_t* cs;
                o_side(ed, v, &cs);
                for (j = 0; j < ed->ncols; j++)
                    probe_sec += o_sectors(alive, n, t[v].dtypes[cs[j]] == 0 ? 4 : 8);
#pragma omp parallel for schedule(static)
                for (int64_t r = 0; r < n; r++) {
                    if (!alive[r]) continue;
                    if (exact) {
                        o_pair key = o_edge_key(&t[v], ed, v, r);
                        o_pair* s = set[p * n_edges + ine[i]];
                        int64_t sn = set_n[p * n_edges + ine[i]];
                        alive[r] = sn > 0 && bsearch(&key, s, (size_t)sn, sizeof(o_pair), o_pair_cmp) != NULL;
                    } else {
                        uint64_t h = o_edge_hash(&t[v], ed, v, r, cfg->seed);
                        alive[r] = (unsigned char)o_filter_probe(filt[p * n_edges + ine[i]],
                                                                 nblocks[p * n_edges + ine[i]], B, K, h);
                    }
                }
            }

            /* survivor bitmap, one word per 32 rows, tail bits zero */
#pragma omp parallel for schedule(static) reduction(+ : c)
            for (int64_t w = 0; w < (n + 31) / 32; w++) {
                uint32_t x = 0;
                for (int64_t r = 32 * w; r < 32 * w + 32 && r < n; r++)
                    if (alive[r]) { x |= 1u << (r & 31); c++; }
                out[w] = x;
            }
            count[p * n_tables + v] = c;

            /* build one fresh outgoing filter per outgoing edge from the survivors' keys */
            int32_t seen_cols[64];
            int32_t n_seen = 0;
            for (i = 0; i < n_edges; i++) {
                int32_t from = p == 0 ? src[i] : dst[i];
                if (from != v || !o_active(e, src, dst, p, i)) continue;
                const o_edge* ed = &e[i];
                const int32_t* cs;
                o_side(ed, v, &cs);
                for (j = 0; j < ed->ncols; j++) {
                    int32_t k2, dup = 0;
                    for (k2 = 0; k2 < n_seen; k2++) dup |= seen_cols[k2] == cs[j];
                    if (!dup && n_seen < 64) {
                        seen_cols[n_seen++] = cs[j];
                        build_sec += o_sectors(alive, n, t[v].dtypes[cs[j]] == 0 ? 4 : 8);
                    }
                }
                int32_t other = ed->t0 == v ? ed->t1 : ed->t0;
                if (exact) {
                    o_pair* s = (o_pair*)malloc(sizeof(o_pair) * (size_t)(c > 0 ? c : 1));
                    int64_t m = 0;
                    for (int64_t r = 0; r < n; r++)
                        if (alive[r]) s[m++] = o_edge_key(&t[v], ed, v, r);
                    qsort(s, (size_t)m, sizeof(o_pair), o_pair_cmp);
                    set[p * n_edges + i] = s;
                    set_n[p * n_edges + i] = m;
                    nblocks[p * n_edges + i] = 0;
                } else {
                    int64_t nb = o_nblocks(c, n_rows[other], cfg->bits_per_key, B);
                    uint32_t* f = filt[p * n_edges + i];
                    memset(f, 0, sizeof(uint32_t) * (size_t)(nb * wpb));
#pragma omp parallel for schedule(static)
                    for (int64_t r = 0; r < n; r++)
                        if (alive[r]) o_filter_insert(f, nb, B, K, o_edge_hash(&t[v], ed, v, r, cfg->seed));
                    nblocks[p * n_edges + i] = nb;
                }
            }
            if (sectors) {
                sectors[(p * n_tables + v) * 2 + 0] = probe_sec;
                sectors[(p * n_tables + v) * 2 + 1] = build_sec;
            }
            free(alive);
        }
    }
    for (i = 0; i < 2 * n_edges; i++) free(set[i]);
    free(set); free(set_n); free(n_rows); free(src); free(dst); free(order); free(ine); free(lvl);
    return 0;
}

/*
 * o_one_hop: the Bloom join (Section 2.1; the BloomJoin baseline of Section
 * 4), a one-hop transfer in one direction.  Every edge has one building
 * table: the smaller one by the transfer graph's orientation (a Bloom join
 * builds on the smaller table), or t0 for a one-way edge.  Its filter holds
 * the join keys of the building table's selected rows -- its local predicate
 * alone, nothing received from another table -- and is sized by the same
 * rule as a transfer's, with c = the number of selected rows.  A table then
 * keeps a selected row iff every filter built for it accepts the row's key.
 *
 * surv[v] (caller-owned, ceil(n_v/32) words), count[v]: the result per
 * table.  filt[e] (Bloom mode; caller-owned, as in o_transfer), nblocks[e]:
 * the filter of edge e (0 blocks in exact mode, where it is the key set).
 * Returns 0, or -1 on invalid input.
 */
int o_one_hop(int32_t n_tables, const o_table* t, int32_t n_edges, const o_edge* e,
              const o_cfg* cfg, int32_t exact, uint32_t* const* surv, int64_t* count,
              uint32_t* const* filt, int64_t* nblocks) {
    int32_t B = cfg->block_bits, K = cfg->k, wpb = cfg->block_bits / 32;
    int32_t v, i;
    if (!o_valid(n_tables, n_edges, e, cfg)) return -1;

    int64_t* n_rows = (int64_t*)calloc((size_t)(n_tables > 0 ? n_tables : 1), sizeof(int64_t));
    int32_t* src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_edges + 1));
    int32_t* dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_edges + 1));
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_tables + 1));
    int32_t* bld = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_edges + 1));
    o_pair** set = (o_pair**)calloc((size_t)(n_edges + 1), sizeof(o_pair*));
    int64_t* set_n = (int64_t*)calloc((size_t)(n_edges + 1), sizeof(int64_t));
    for (v = 0; v < n_tables; v++) n_rows[v] = t[v].n_rows;
    o_orient(n_tables, n_rows, n_edges, e, src, dst, order);

    /* build: one filter per edge from the building table's selected rows */
    for (i = 0; i < n_edges; i++) {
        const o_edge* ed = &e[i];
        int32_t b = (ed->flags & O_EDGE_ONE_WAY) ? ed->t0 : src[i];
        int32_t q = b == ed->t0 ? ed->t1 : ed->t0;
        int64_t n = n_rows[b], c = 0, r;
        bld[i] = b;
        for (r = 0; r < n; r++) c += t[b].sel ? o_bit(t[b].sel, r) : 1;
        if (exact) {
            o_pair* s = (o_pair*)malloc(sizeof(o_pair) * (size_t)(c > 0 ? c : 1));
            int64_t m = 0;
            for (r = 0; r < n; r++)
                if (!t[b].sel || o_bit(t[b].sel, r)) s[m++] = o_edge_key(&t[b], ed, b, r);
            qsort(s, (size_t)m, sizeof(o_pair), o_pair_cmp);
            set[i] = s;
            set_n[i] = m;
            nblocks[i] = 0;
        } else {
            int64_t nb = o_nblocks(c, n_rows[q], cfg->bits_per_key, B);
            memset(filt[i], 0, sizeof(uint32_t) * (size_t)(nb * wpb));
#pragma omp parallel for schedule(static)
            for (r = 0; r < n; r++)
                if (!t[b].sel || o_bit(t[b].sel, r)) o_filter_insert(filt[i], nb, B, K, o_edge_hash(&t[b], ed, b, r, cfg->seed));
            nblocks[i] = nb;
        }
    }

    /* probe: a selected row survives iff every filter built for its table accepts its key */
    for (v = 0; v < n_tables; v++) {
        int64_t n = n_rows[v], c = 0, w;
        unsigned char* alive = (unsigned char*)malloc((size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < n; r++) alive[r] = t[v].sel ? (unsigned char)o_bit(t[v].sel, r) : 1;
        for (i = 0; i < n_edges; i++) {
            const o_edge* ed = &e[i];
            if (bld[i] == v || (ed->t0 != v && ed->t1 != v)) continue;
#pragma omp parallel for schedule(static)
            for (int64_t r = 0; r < n; r++) {
                if (!alive[r]) continue;
                if (exact) {
                    o_pair key = o_edge_key(&t[v], ed, v, r);
                    alive[r] = set_n[i] > 0 && bsearch(&key, set[i], (size_t)set_n[i], sizeof(o_pair), o_pair_cmp) != NULL;
                } else {
                    alive[r] = (unsigned char)o_filter_probe(filt[i], nblocks[i], B, K, o_edge_hash(&t[v], ed, v, r, cfg->seed));
                }
            }
        }
#pragma omp parallel for schedule(static) reduction(+ : c)
        for (w = 0; w < (n + 31) / 32; w++) {
            uint32_t x = 0;
            for (int64_t r = 32 * w; r < 32 * w + 32 && r < n; r++)
                if (alive[r]) { x |= 1u << (r & 31); c++; }
            surv[v][w] = x;
        }
        count[v] = c;
        free(alive);
    }
    for (i = 0; i < n_edges; i++) free(set[i]);
    free(set); free(set_n); free(n_rows); free(src); free(dst); free(order); free(bld);
    return 0;
}

/* ---- join phase: the size of the join (Section 3.3) ------------------- */

typedef struct { uint64_t a, b, w; } o_kw;

static int o_kw_cmp(const void* x, const void* y) {
    const o_kw* p = (const o_kw*)x;
    const o_kw* q = (const o_kw*)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

/*
 * o_join_count: the number of tuples in the join of the rows of every
 * table whose bit is set in rows[v] (caller-owned bitmaps, ceil(n_v/32)
 * words; NULL = every row), for an acyclic join graph (a forest) of inner
 * equi-joins.  Each tree is rooted at its largest table (ties: higher id),
 * and in post-order every table's row weight (1 for a set row, else 0) is
 * multiplied, for each child, by the summed weights of the child's rows
 * with an equal key on the edge joining them; a tree's count is its root's
 * weight sum, and the join's is the product over trees.  Returns 0 and the
 * count (mod 2^64) at *out, -1 on invalid input, -2 if the graph has a cycle
 * or a one-way edge.
 */
int o_join_count(int32_t n_tables, const o_table* t, int32_t n_edges, const o_edge* e,
                 uint32_t* const* rows, uint64_t* out) {
    int32_t v, i;
    if (n_tables < 1) return -1;
    for (i = 0; i < n_edges; i++) {
        if (e[i].ncols < 1 || e[i].ncols > 2 || e[i].t0 == e[i].t1) return -1;
        if (e[i].t0 < 0 || e[i].t0 >= n_tables || e[i].t1 < 0 || e[i].t1 >= n_tables) return -1;
        if (e[i].flags) return -2;
    }
    /* cycle check (union-find) */
    int32_t* uf = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_tables);
    for (v = 0; v < n_tables; v++) uf[v] = v;
    for (i = 0; i < n_edges; i++) {
        int32_t a = e[i].t0, b = e[i].t1;
        while (uf[a] != a) a = uf[a];
        while (uf[b] != b) b = uf[b];
        if (a == b) { free(uf); return -2; }
        uf[a] = b;
    }
    /* weights */
    uint64_t** wt = (uint64_t**)malloc(sizeof(uint64_t*) * (size_t)n_tables);
    for (v = 0; v < n_tables; v++) {
        int64_t n = t[v].n_rows;
        wt[v] = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t r = 0; r < n; r++)
            wt[v][r] = (!rows || !rows[v]) ? 1u : (uint64_t)((rows[v][r >> 5] >> (r & 31)) & 1u);
    }
    /* roots: the largest table of each component; parent links by DFS */
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_tables);
    int32_t* pedge = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_tables);
    int32_t* post = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_tables);
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_tables);
    unsigned char* seen = (unsigned char*)calloc((size_t)n_tables, 1);
    int32_t n_post = 0;
    uint64_t total = 1;
    for (;;) {
        int32_t root = -1;
        for (v = 0; v < n_tables; v++)
            if (!seen[v] && (root < 0 || t[v].n_rows >= t[root].n_rows)) root = v;
        if (root < 0) break;
        /* iterative DFS: order[] lists the tree top-down; reversed it is a post-order */
        int32_t sp = 0, first = n_post;
        stack[sp++] = root;
        seen[root] = 1;
        parent[root] = -1;
        pedge[root] = -1;
        while (sp) {
            int32_t x = stack[--sp];
            post[n_post++] = x;
            for (i = 0; i < n_edges; i++) {
                int32_t y = e[i].t0 == x ? e[i].t1 : (e[i].t1 == x ? e[i].t0 : -1);
                if (y < 0 || seen[y]) continue;
                seen[y] = 1;
                parent[y] = x;
                pedge[y] = i;
                stack[sp++] = y;
            }
        }
        /* children before parents */
        for (int32_t j = n_post - 1; j > first; j--) {
            int32_t c = post[j], p = parent[c];
            const o_edge* ed = &e[pedge[c]];
            int64_t nc = t[c].n_rows, np = t[p].n_rows, m = 0;
            o_kw* kw = (o_kw*)malloc(sizeof(o_kw) * (size_t)(nc > 0 ? nc : 1));
            for (int64_t r = 0; r < nc; r++) {
                if (!wt[c][r]) continue;
                o_pair k = o_edge_key(&t[c], ed, c, r);
                kw[m].a = k.a; kw[m].b = k.b; kw[m].w = wt[c][r];
                m++;
            }
            qsort(kw, (size_t)m, sizeof(o_kw), o_kw_cmp);
            /* sum the weights of equal keys into the first of each run */
            int64_t u = 0;
            for (int64_t r = 0; r < m; r++) {
                if (u > 0 && kw[u - 1].a == kw[r].a && kw[u - 1].b == kw[r].b) kw[u - 1].w += kw[r].w;
                else kw[u++] = kw[r];
            }
            for (int64_t r = 0; r < np; r++) {
                if (!wt[p][r]) continue;
                o_pair k = o_edge_key(&t[p], ed, p, r);
                o_kw probe = {k.a, k.b, 0};
                o_kw* hit = u > 0 ? (o_kw*)bsearch(&probe, kw, (size_t)u, sizeof(o_kw), o_kw_cmp) : NULL;
                wt[p][r] *= hit ? hit->w : 0u;
            }
            free(kw);
        }
        uint64_t s = 0;
        for (int64_t r = 0; r < t[root].n_rows; r++) s += wt[root][r];
        total *= s;
    }
    for (v = 0; v < n_tables; v++) free(wt[v]);
    free(wt); free(uf); free(parent); free(pedge); free(post); free(stack); free(seen);
    *out = total;
    return 0;
}
