/*
 * Oracle for the bit-adaptive particle position compressor of
 * Ren, Di, Zhang, Zhao, Guo, "An Error-Bounded Lossy Compression Method with
 * Bit-Adaptive Quantization for Particle Data" (arXiv 2404.02826).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow CPU restatement of the
 * method, in double precision, written to check the CUDA library against.
 * Compiled as usual it is single-threaded.  The same source compiled with
 * -fopenmp runs its independent loops in parallel (particles in the range
 * and quantization, the two halves of every split, leaves in the bit boxes,
 * the packing and the decoding); every particle's arithmetic and every
 * output byte are the same, and the leaves are listed in the same order.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
 * legs of bench.py load it; the product path never calls it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Steps, in the paper's order (section / equation in brackets):
 *   1. error bound eps and lattice step s   [Sec. 3, absolute / relative bound]
 *   2. quantization onto the 2*eb lattice   [Sec. 3, linear-scale quantization, Eq. 1]
 *   3. median k-d partition, leaves <= r    [Sec. 4.1, initial particle partitioning]
 *   4. bit box per leaf: AABB, centre, m_d  [Sec. 4.1, bit box construction, Eq. 2]
 *   5. codes and the sequence layout        [Fig. 2 caption; Sec. 4.2, Fig. 4]
 *   6. decoding                             [Sec. 3, dequantization]
 *   7. NRMSE / PSNR                         [Sec. 5.1]
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - the lattice origin is the per-axis minimum and the step is s = 2*eb',
 *     eb' = eps - ulp_T(M2) - 4*ulp_f64(M2), M2 = 2*max(max|p|, eps), so that the
 *     bound survives the rounding of the reconstruction to the input type;
 *     when every particle is identical (Delta_max = 0) the step is 1;
 *   - q = rint(((double)p - o) / s), round-half-even, one division, no
 *     reciprocal; codes must stay below 2^30;
 *   - the split axis is depth mod 3; a node is split on the total order
 *     (code on the axis, original index); the first floor(n/2) go left, so the
 *     median goes to the larger-coordinate side (Sec. 4.1);
 *   - the bit-box centre is the leaf particle minimising the squared lattice
 *     distance to the AABB centre, first in leaf order on ties;
 *   - a zero minimum or maximum is taken as +0 (signed zeros compare equal);
 *   - the centre is stored as its lattice code (not as a lossless float) and the
 *     particle count replaces the end mark; see the stream layout below;
 *   - lossless axes (Sec. 4.1: a dimension whose m_d exceeds M is stored as the
 *     original coordinates): codes here stay below 2^30 (m_d <= 31), so an axis
 *     whose code range reaches 2^30, or every axis when no lattice meets eps
 *     within the type's resolution (eb' <= 0), is stored losslessly in every
 *     leaf; the tree splits such an axis on the key
 *     floor((p - lo) / (hi - lo) * 2^29), monotone in the coordinate.
 *
 * Precision: compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NONFINITE 2
#define OR_ERR_EB_TOO_SMALL 3
#define OR_ERR_RANGE 4
#define OR_ERR_CAPACITY 5
#define OR_ERR_CORRUPT 6
#define OR_ERR_NOMEM 9

#define OR_F32 0
#define OR_F64 1
#define OR_ABS 0
#define OR_REL 1

#define OR_CODE_LIMIT (1LL << 30) /* codes must be < 2^30, so m_d <= 31 */
#define OR_RAW_KEY_TOP 536870912.0 /* 2^29: largest split key of a lossless axis */
#define OR_HEADER_BYTES 96u
#define OR_LEAF_BYTES 32u

/* ------------------------------------------------------------------------ */
/* Step 1: error bound and lattice (Sec. 3).                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    double lo[3], hi[3];  /* per-axis min / max of the input                    */
    double delta_max;     /* Delta_max: largest per-axis range (Sec. 3)          */
    double eps;           /* absolute bound: eb (abs) or eb * Delta_max (rel)    */
    double eb_prime;      /* eps minus the rounding margin                        */
    double s;             /* lattice step = 2 * eb'                               */
    double o[3];          /* lattice origin = per-axis minimum                    */
    int64_t qmax[3];      /* largest code per axis (split key of a lossless axis) */
    uint32_t raw;         /* bit d: axis d stored losslessly (Sec. 4.1, m_d > M)   */
    int raw_cause;        /* why: OR_ERR_EB_TOO_SMALL (no lattice) or OR_ERR_RANGE  */
} oracle_bound;

static double coord(const void *pos, int dtype, uint64_t i, int d)
{
    if (dtype == OR_F32) return (double)((const float *)pos)[3 * i + d];
    return ((const double *)pos)[3 * i + d];
}

/* Spacing of the floating-point grid with `prec` significand bits at the
 * magnitude of x > 0 (subnormal spacing below 2^emin). */
static double grid_spacing(double x, int prec, int emin)
{
    int e;
    (void)frexp(x, &e); /* x = f * 2^e, f in [0.5, 1) */
    int ex = e - 1;     /* floor(log2 x) */
    if (ex < emin) ex = emin;
    return ldexp(1.0, ex - (prec - 1));
}

/* Quantization code of one coordinate: index of the 2*eb' interval that holds
 * it, counted from the origin (Sec. 3, Eq. 1 with the prediction at o). */
static int64_t quantize_one(double p, double o, double s)
{
    double t = (p - o) / s;
    return (int64_t)nearbyint(t);
}

/* Split key of a coordinate on a lossless axis: its place in [lo, hi] on a
 * grid of 2^29 steps (monotone in p; the coordinate itself is stored). */
static int64_t raw_key(double p, double lo, double hi)
{
    double span = hi - lo;
    if (!(span > 0.0)) return 0;
    double t = floor(((p - lo) / span) * OR_RAW_KEY_TOP);
    if (t < 0.0) t = 0.0;
    if (t > OR_RAW_KEY_TOP) t = OR_RAW_KEY_TOP;
    return (int64_t)t;
}

int oracle_error_bound(const void *pos, uint64_t n, int dtype, int eb_mode, double eb,
                       oracle_bound *b)
{
    if (dtype != OR_F32 && dtype != OR_F64) return OR_ERR_ARG;
    if (eb_mode != OR_ABS && eb_mode != OR_REL) return OR_ERR_ARG;
    if (!(eb > 0.0) || !isfinite(eb)) return OR_ERR_ARG;
    if (n > 0 && pos == NULL) return OR_ERR_ARG;
    memset(b, 0, sizeof(*b));
    b->s = 1.0;
    if (n == 0) {
        b->eps = (eb_mode == OR_ABS) ? eb : 0.0;
        b->eb_prime = b->eps;
        return OR_OK;
    }
    double lo0 = INFINITY, lo1 = INFINITY, lo2 = INFINITY, hi0 = -INFINITY, hi1 = -INFINITY, hi2 = -INFINITY;
    int bad = 0;
#pragma omp parallel for reduction(min : lo0, lo1, lo2) reduction(max : hi0, hi1, hi2) reduction(| : bad)
    for (uint64_t i = 0; i < n; i++) {
        double x = coord(pos, dtype, i, 0), y = coord(pos, dtype, i, 1), z = coord(pos, dtype, i, 2);
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) bad = 1;
        if (x < lo0) lo0 = x;
        if (x > hi0) hi0 = x;
        if (y < lo1) lo1 = y;
        if (y > hi1) hi1 = y;
        if (z < lo2) lo2 = z;
        if (z > hi2) hi2 = z;
    }
    if (bad) return OR_ERR_NONFINITE;
    b->lo[0] = lo0;
    b->lo[1] = lo1;
    b->lo[2] = lo2;
    b->hi[0] = hi0;
    b->hi[1] = hi1;
    b->hi[2] = hi2;
    /* A zero extremum is taken as +0, so that the result does not depend on
     * whether -0 or +0 was met first. */
    for (int d = 0; d < 3; d++) {
        if (b->lo[d] == 0.0) b->lo[d] = 0.0;
        if (b->hi[d] == 0.0) b->hi[d] = 0.0;
    }
    /* Delta_max: the maximum range of coordinates across all dimensions. */
    b->delta_max = 0.0;
    for (int d = 0; d < 3; d++) {
        double r = b->hi[d] - b->lo[d];
        if (r > b->delta_max) b->delta_max = r;
    }
    b->eps = (eb_mode == OR_ABS) ? eb : eb * b->delta_max;
    for (int d = 0; d < 3; d++) b->o[d] = b->lo[d];
    if (b->delta_max == 0.0) { /* every particle identical: all codes are 0 */
        b->eb_prime = b->eps;
        b->s = 1.0;
        return OR_OK;
    }
    double m = 0.0;
    for (int d = 0; d < 3; d++) {
        if (fabs(b->lo[d]) > m) m = fabs(b->lo[d]);
        if (fabs(b->hi[d]) > m) m = fabs(b->hi[d]);
    }
    double m2 = 2.0 * (m > b->eps ? m : b->eps);
    double tmax = (dtype == OR_F32) ? (double)FLT_MAX : DBL_MAX;
    if (!(m2 <= tmax)) return OR_ERR_RANGE;
    double ulp_t = (dtype == OR_F32) ? grid_spacing(m2, 24, -126) : grid_spacing(m2, 53, -1022);
    double ulp_d = grid_spacing(m2, 53, -1022);
    b->eb_prime = b->eps - ulp_t - 4.0 * ulp_d;
    if (!(b->eb_prime > 0.0)) {
        /* No lattice keeps the bound through the rounding to the type: every
         * axis is stored losslessly (the step is then unused and 1). */
        b->raw = 7u;
        b->raw_cause = OR_ERR_EB_TOO_SMALL;
        b->s = 1.0;
    } else {
        b->s = 2.0 * b->eb_prime;
        for (int d = 0; d < 3; d++) {
            b->qmax[d] = quantize_one(b->hi[d], b->o[d], b->s);
            if (b->qmax[d] >= OR_CODE_LIMIT) { /* wider than the codes: this axis losslessly */
                b->raw |= 1u << d;
                b->raw_cause = OR_ERR_RANGE;
            }
        }
    }
    for (int d = 0; d < 3; d++)
        if (b->raw & (1u << d)) b->qmax[d] = raw_key(b->hi[d], b->lo[d], b->hi[d]);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 2: quantization (Sec. 3).                                            */
/* ------------------------------------------------------------------------ */

int oracle_quantize(const void *pos, uint64_t n, int dtype, const oracle_bound *b, int64_t *q)
{
#pragma omp parallel for
    for (uint64_t i = 0; i < n; i++)
        for (int d = 0; d < 3; d++)
            q[3 * i + d] = (b->raw & (1u << d)) ? raw_key(coord(pos, dtype, i, d), b->lo[d], b->hi[d])
                                                 : quantize_one(coord(pos, dtype, i, d), b->o[d], b->s);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 3: median k-d partition (Sec. 4.1).                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t key;
    uint64_t idx;
} keyed;

static int by_key_then_index(const void *a, const void *b)
{
    const keyed *x = (const keyed *)a, *y = (const keyed *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

static int by_index(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

typedef struct {
    uint64_t *leaf_off, *leaf_cnt;
    uint64_t num_leaves, cap;
} leaf_list;

static int leaf_push(leaf_list *l, uint64_t off, uint64_t cnt)
{
    if (l->num_leaves == l->cap) {
        uint64_t nc = l->cap ? 2 * l->cap : 64;
        uint64_t *a = realloc(l->leaf_off, nc * sizeof(uint64_t));
        if (!a) return OR_ERR_NOMEM;
        l->leaf_off = a;
        uint64_t *c = realloc(l->leaf_cnt, nc * sizeof(uint64_t));
        if (!c) return OR_ERR_NOMEM;
        l->leaf_cnt = c;
        l->cap = nc;
    }
    l->leaf_off[l->num_leaves] = off;
    l->leaf_cnt[l->num_leaves] = cnt;
    l->num_leaves++;
    return OR_OK;
}

/* ids[0..cnt) holds the node's particles in increasing original index.  A node
 * with at most r particles is a subregion (leaf).  Otherwise the node is split
 * by the median on its axis: sorting the node by (code, index), the first
 * floor(cnt/2) particles form the left child, so the median itself lies on the
 * side with larger coordinates.  Both children keep index order.  The two
 * children own disjoint ranges of ids, so they may be ordered at once.
 * The axis is depth mod 3 (rule 0), or (rule 1) the axis of the node's widest
 * cell: the root's cell spans codes [0, max code] per axis, and a split at
 * median code v gives the left child the cell up to v and the right child the
 * cell from v on that axis; equal widths go to the lowest axis. */
typedef struct {
    int64_t lo[3], hi[3];
} cell;

static int split_node(const int64_t *q, uint64_t *ids, uint64_t base, uint64_t cnt, int depth, uint64_t r, int rule,
                      cell box)
{
    if (cnt <= r) return OR_OK;
    int axis = depth % 3;
    if (rule == 1) {
        axis = 0;
        for (int d = 1; d < 3; d++)
            if (box.hi[d] - box.lo[d] > box.hi[axis] - box.lo[axis]) axis = d;
    }
    keyed *tmp = malloc(cnt * sizeof(keyed));
    if (!tmp) return OR_ERR_NOMEM;
    for (uint64_t i = 0; i < cnt; i++) {
        tmp[i].key = q[3 * ids[base + i] + axis];
        tmp[i].idx = ids[base + i];
    }
    qsort(tmp, cnt, sizeof(keyed), by_key_then_index);
    uint64_t k = cnt / 2;
    int64_t v = tmp[k].key; /* the median code */
    for (uint64_t i = 0; i < cnt; i++) ids[base + i] = tmp[i].idx;
    free(tmp);
    cell left = box, right = box;
    left.hi[axis] = v;
    right.lo[axis] = v;
    qsort(ids + base, k, sizeof(uint64_t), by_index);
    qsort(ids + base + k, cnt - k, sizeof(uint64_t), by_index);
    int rc_left = OR_OK, rc_right = OR_OK;
#pragma omp task shared(rc_left) if (cnt > 65536)
    rc_left = split_node(q, ids, base, k, depth + 1, r, rule, left);
    rc_right = split_node(q, ids, base + k, cnt - k, depth + 1, r, rule, right);
#pragma omp taskwait
    return rc_left ? rc_left : rc_right;
}

/* The subregions of the same recursion, left to right: they depend only on the
 * node sizes, floor(cnt/2) and the rest. */
static int collect_leaves(uint64_t base, uint64_t cnt, uint64_t r, leaf_list *leaves)
{
    if (cnt <= r) return leaf_push(leaves, base, cnt);
    uint64_t k = cnt / 2;
    int rc = collect_leaves(base, k, r, leaves);
    if (rc) return rc;
    return collect_leaves(base + k, cnt - k, r, leaves);
}

/* order[0..n): original indices, leaves concatenated left to right.
 * leaf_off / leaf_cnt: allocated here (free with oracle_free). */
int oracle_kdtree_rule(const int64_t *q, uint64_t n, uint64_t r, int rule, uint64_t *order, uint64_t **leaf_off,
                       uint64_t **leaf_cnt, uint64_t *num_leaves)
{
    if (r < 1 || rule < 0 || rule > 1) return OR_ERR_ARG;
    leaf_list l = {0};
    for (uint64_t i = 0; i < n; i++) order[i] = i;
    int rc = OR_OK;
    if (n > 0) {
        cell root;
        for (int d = 0; d < 3; d++) {
            root.lo[d] = 0;
            root.hi[d] = 0;
        }
        for (uint64_t i = 0; i < n; i++)
            for (int d = 0; d < 3; d++)
                if (q[3 * i + d] > root.hi[d]) root.hi[d] = q[3 * i + d];
#pragma omp parallel
#pragma omp single
        rc = split_node(q, order, 0, n, 0, r, rule, root);
        if (!rc) rc = collect_leaves(0, n, r, &l);
    }
    if (rc) {
        free(l.leaf_off);
        free(l.leaf_cnt);
        return rc;
    }
    *leaf_off = l.leaf_off;
    *leaf_cnt = l.leaf_cnt;
    *num_leaves = l.num_leaves;
    return OR_OK;
}

int oracle_kdtree(const int64_t *q, uint64_t n, uint64_t r, uint64_t *order, uint64_t **leaf_off,
                  uint64_t **leaf_cnt, uint64_t *num_leaves)
{
    return oracle_kdtree_rule(q, n, r, 0, order, leaf_off, leaf_cnt, num_leaves);
}

/* ------------------------------------------------------------------------ */
/* Step 4: bit box of one leaf (Sec. 4.1, Eq. 2).                            */
/* ------------------------------------------------------------------------ */

/* Eq. 2 on the lattice.  With positions on the lattice the distance from the
 * centre is D = s*R and 2*eb' = s, so Eq. 2 reads m = ceil(log2(R + 0.5) + 1).
 * For R = 0 that is 0.  For R >= 1 it is the least m with 2^(m-1) - 1 >= R,
 * i.e. the bit length of R plus one. */
uint32_t oracle_num_bits(uint64_t R)
{
    if (R == 0) return 0;
    uint32_t m = 1;
    while (((1ULL << (m - 1)) - 1ULL) < R) m++;
    return m;
}

/* leafq[0..n) x 3 codes of one leaf in leaf order.  Outputs: centre position in
 * the leaf, the AABB, the centre code and m_d. */
int oracle_bitbox(const int64_t *leafq, uint64_t n, uint64_t *centre, int64_t lo[3], int64_t hi[3],
                  int64_t qref[3], uint32_t m[3])
{
    if (n == 0) return OR_ERR_ARG;
    for (int d = 0; d < 3; d++) lo[d] = hi[d] = leafq[d];
    for (uint64_t i = 1; i < n; i++)
        for (int d = 0; d < 3; d++) {
            if (leafq[3 * i + d] < lo[d]) lo[d] = leafq[3 * i + d];
            if (leafq[3 * i + d] > hi[d]) hi[d] = leafq[3 * i + d];
        }
    /* The centre is the particle closest to the AABB centre (lo+hi)/2; in
     * doubled lattice units the squared distance is an exact integer. */
    uint64_t best = 0, best_d2 = UINT64_MAX;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t d2 = 0;
        for (int d = 0; d < 3; d++) {
            int64_t t = 2 * leafq[3 * i + d] - lo[d] - hi[d];
            d2 += (uint64_t)(t * t);
        }
        if (d2 < best_d2) {
            best_d2 = d2;
            best = i;
        }
    }
    *centre = best;
    for (int d = 0; d < 3; d++) {
        qref[d] = leafq[3 * best + d];
        int64_t a = qref[d] - lo[d], c = hi[d] - qref[d];
        uint64_t R = (uint64_t)(a > c ? a : c);
        m[d] = oracle_num_bits(R);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 5: stream layout (Sec. 4.2, Fig. 4; Fig. 2 caption for the codes).   */
/*                                                                          */
/* Header, 96 bytes, little-endian:                                          */
/*   0 "PCB1"  4 u16 version=1  6 u8 dtype  7 u8 eb_mode  8 u64 n             */
/*   16 f64 eb as given  24 f64 eps  32 f64 s  40 f64 o[3]                    */
/*   64 u64 num_leaves  72 u64 payload_words  80 u32 leaf_size                 */
/*   84 u8 lossless-axis mask (bit d: axis d)  85..95 zero                     */
/* Leaf table, 32 bytes per sequence (leaf), in leaf order:                  */
/*   0 u64 first output particle  8 u64 first payload word                   */
/*   16 i32 q_ref[3] (centre code)  28 u8 m[3]  31 u8 zero                    */
/* Payload: u32 words.  Each leaf starts on a fresh word; its non-centre      */
/* particles follow in leaf order, each as c_x (m_x bits), c_y, c_z, packed   */
/* least-significant bit first.  c_d = (q_d - q_ref_d) + 2^(m_d-1) - 1.        */
/* With a nonzero lossless-axis mask every leaf lists all its particles, the   */
/* centre first, then the rest in leaf order; a lossless axis has m_d = M      */
/* (32 or 64) and q_ref_d = 0, and its field is the coordinate's M-bit pattern. */
/* ------------------------------------------------------------------------ */

static void put_u16(uint8_t *p, uint16_t v)
{
    p[0] = (uint8_t)v;
    p[1] = (uint8_t)(v >> 8);
}
static void put_u32(uint8_t *p, uint32_t v)
{
    for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void put_u64(uint8_t *p, uint64_t v)
{
    for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void put_f64(uint8_t *p, double v)
{
    uint64_t u;
    memcpy(&u, &v, 8);
    put_u64(p, u);
}
static uint16_t get_u16(const uint8_t *p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t get_u32(const uint8_t *p)
{
    uint32_t v = 0;
    for (int i = 0; i < 4; i++) v |= (uint32_t)p[i] << (8 * i);
    return v;
}
static uint64_t get_u64(const uint8_t *p)
{
    uint64_t v = 0;
    for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i);
    return v;
}
static double get_f64(const uint8_t *p)
{
    uint64_t u = get_u64(p);
    double v;
    memcpy(&v, &u, 8);
    return v;
}

/* Append `nbits` low bits of `v` to the word array, least significant first. */
static void write_bits(uint32_t *words, uint64_t *bitpos, uint64_t v, uint32_t nbits)
{
    for (uint32_t b = 0; b < nbits; b++) {
        uint64_t pos = *bitpos + b;
        if ((v >> b) & 1ULL) words[pos >> 5] |= 1u << (pos & 31);
    }
    *bitpos += nbits;
}

static uint64_t read_bits(const uint32_t *words, uint64_t bitpos, uint32_t nbits)
{
    uint64_t v = 0;
    for (uint32_t b = 0; b < nbits; b++) {
        uint64_t pos = bitpos + b;
        if ((words[pos >> 5] >> (pos & 31)) & 1u) v |= 1ULL << b;
    }
    return v;
}

/* Number of leaves the partition produces, for sizing. */
static uint64_t leaves_for(uint64_t n, uint64_t r)
{
    if (n == 0) return 0;
    if (n <= r) return 1;
    return leaves_for(n / 2, r) + leaves_for(n - n / 2, r);
}

/* Full compression.  On success *out (malloc'd) holds the stream and *perm
 * (malloc'd, may be NULL on request) maps each decoded particle to its
 * original index. */
int oracle_compress_rule(const void *pos, uint64_t n, int dtype, int eb_mode, double eb, uint64_t leaf_size,
                         int rule, uint8_t **out, uint64_t *out_bytes, uint64_t **perm_out)
{
    *out = NULL;
    *out_bytes = 0;
    if (perm_out) *perm_out = NULL;
    if (leaf_size < 1) return OR_ERR_ARG;
    oracle_bound b;
    int rc = oracle_error_bound(pos, n, dtype, eb_mode, eb, &b);
    if (rc) return rc;

    int64_t *q = NULL;
    uint64_t *order = NULL, *loff = NULL, *lcnt = NULL, *perm = NULL, nl = 0;
    uint64_t *centre = NULL, *wofs = NULL;
    int64_t *qref = NULL;
    uint32_t *mm = NULL, *words = NULL;
    uint8_t *buf = NULL;
    rc = OR_ERR_NOMEM;

    q = malloc((n ? n : 1) * 3 * sizeof(int64_t));
    order = malloc((n ? n : 1) * sizeof(uint64_t));
    perm = malloc((n ? n : 1) * sizeof(uint64_t));
    if (!q || !order || !perm) goto done;
    oracle_quantize(pos, n, dtype, &b, q);
    rc = oracle_kdtree_rule(q, n, leaf_size, rule, order, &loff, &lcnt, &nl);
    if (rc) goto done;
    rc = OR_ERR_NOMEM;

    centre = malloc((nl ? nl : 1) * sizeof(uint64_t));
    wofs = malloc((nl ? nl : 1) * sizeof(uint64_t));
    qref = malloc((nl ? nl : 1) * 3 * sizeof(int64_t));
    mm = malloc((nl ? nl : 1) * 3 * sizeof(uint32_t));
    if (!centre || !wofs || !qref || !mm) goto done;
    /* Bit boxes, and the size of each leaf's code block: storage-cost term (3)
     * of Sec. 4.2, (m_x + m_y + m_z)(n_s - 1) bits, rounded up to words. */
    uint64_t maxleaf = leaf_size < n ? leaf_size : n;
    int nomem = 0;
#pragma omp parallel reduction(| : nomem)
    {
        int64_t *leafq = malloc((maxleaf ? maxleaf : 1) * 3 * sizeof(int64_t));
        if (!leafq) nomem = 1;
#pragma omp for schedule(dynamic, 16)
        for (uint64_t L = 0; L < nl; L++) {
            if (!leafq) continue;
            for (uint64_t i = 0; i < lcnt[L]; i++)
                for (int d = 0; d < 3; d++) leafq[3 * i + d] = q[3 * order[loff[L] + i] + d];
            int64_t lo[3], hi[3];
            oracle_bitbox(leafq, lcnt[L], &centre[L], lo, hi, &qref[3 * L], &mm[3 * L]);
        }
        free(leafq);
    }
    if (nomem) goto done;
    /* Lossless axes (Sec. 4.1, m_d > M): M bits of the coordinate for every
     * particle of the leaf, the centre included. */
    const uint32_t M = dtype == OR_F32 ? 32u : 64u;
    for (uint64_t L = 0; L < nl; L++)
        for (int d = 0; d < 3; d++)
            if (b.raw & (1u << d)) {
                mm[3 * L + d] = M;
                qref[3 * L + d] = 0;
            }
    uint64_t total_words = 0;
    for (uint64_t L = 0; L < nl; L++) {
        uint64_t w = (uint64_t)(mm[3 * L] + mm[3 * L + 1] + mm[3 * L + 2]);
        uint64_t bits = b.raw ? w * lcnt[L] : w * (lcnt[L] - 1);
        wofs[L] = total_words;
        total_words += (bits + 31) / 32;
    }

    uint64_t bytes = OR_HEADER_BYTES + OR_LEAF_BYTES * nl + 4 * total_words;
    buf = calloc(bytes, 1);
    if (!buf) goto done;
    memcpy(buf, "PCB1", 4);
    put_u16(buf + 4, 1);
    buf[6] = (uint8_t)dtype;
    buf[7] = (uint8_t)eb_mode;
    put_u64(buf + 8, n);
    put_f64(buf + 16, eb);
    put_f64(buf + 24, b.eps);
    put_f64(buf + 32, b.s);
    for (int d = 0; d < 3; d++) put_f64(buf + 40 + 8 * d, b.o[d]);
    put_u64(buf + 64, nl);
    put_u64(buf + 72, total_words);
    put_u32(buf + 80, (uint32_t)leaf_size);
    buf[84] = (uint8_t)b.raw;
    words = calloc(total_words ? total_words : 1, sizeof(uint32_t));
    if (!words) goto done;

    /* Every leaf owns its words (it starts on a fresh one) and its decoded
     * positions (from its first particle on), so leaves are written apart. */
#pragma omp parallel for schedule(dynamic, 16)
    for (uint64_t L = 0; L < nl; L++) {
        uint8_t *rec = buf + OR_HEADER_BYTES + OR_LEAF_BYTES * L;
        put_u64(rec + 0, loff[L]);
        put_u64(rec + 8, wofs[L]);
        for (int d = 0; d < 3; d++) put_u32(rec + 16 + 4 * d, (uint32_t)(int32_t)qref[3 * L + d]);
        for (int d = 0; d < 3; d++) rec[28 + d] = (uint8_t)mm[3 * L + d];
        /* Decoded order: the centre first, then the rest in leaf order. */
        uint64_t outpos = loff[L];
        perm[outpos++] = order[loff[L] + centre[L]];
        uint64_t bitpos = 32 * wofs[L];
        if (b.raw) {
            /* every particle, the centre first: lossless axes as M-bit patterns */
            for (uint64_t k = 0; k < lcnt[L]; k++) {
                uint64_t i = k == 0 ? centre[L] : (k - 1 < centre[L] ? k - 1 : k);
                uint64_t id = order[loff[L] + i];
                if (k > 0) perm[outpos++] = id;
                for (int d = 0; d < 3; d++) {
                    uint32_t md = mm[3 * L + d];
                    if (b.raw & (1u << d)) {
                        uint64_t bitsval;
                        if (dtype == OR_F32) {
                            uint32_t u;
                            memcpy(&u, (const float *)pos + 3 * id + d, 4);
                            bitsval = u;
                        } else {
                            memcpy(&bitsval, (const double *)pos + 3 * id + d, 8);
                        }
                        write_bits(words, &bitpos, bitsval, md);
                    } else if (md) {
                        int64_t c = (q[3 * id + d] - qref[3 * L + d]) + ((1LL << (md - 1)) - 1);
                        write_bits(words, &bitpos, (uint64_t)c, md);
                    }
                }
            }
            continue;
        }
        for (uint64_t i = 0; i < lcnt[L]; i++) {
            if (i == centre[L]) continue;
            uint64_t id = order[loff[L] + i];
            perm[outpos++] = id;
            for (int d = 0; d < 3; d++) {
                uint32_t md = mm[3 * L + d];
                if (md == 0) continue;
                /* Code of the interval holding the particle: the centre's own
                 * interval is 2^(m-1) - 1 (Fig. 2 caption: one below is 2^(m-1) - 2). */
                int64_t c = (q[3 * id + d] - qref[3 * L + d]) + ((1LL << (md - 1)) - 1);
                write_bits(words, &bitpos, (uint64_t)c, md);
            }
        }
    }
    for (uint64_t w = 0; w < total_words; w++)
        put_u32(buf + OR_HEADER_BYTES + OR_LEAF_BYTES * nl + 4 * w, words[w]);

    *out = buf;
    buf = NULL;
    *out_bytes = bytes;
    if (perm_out) {
        *perm_out = perm;
        perm = NULL;
    }
    rc = OR_OK;
done:
    free(q);
    free(order);
    free(loff);
    free(lcnt);
    free(perm);
    free(centre);
    free(wofs);
    free(qref);
    free(mm);
    free(words);
    free(buf);
    return rc;
}

int oracle_compress(const void *pos, uint64_t n, int dtype, int eb_mode, double eb, uint64_t leaf_size,
                    uint8_t **out, uint64_t *out_bytes, uint64_t **perm_out)
{
    return oracle_compress_rule(pos, n, dtype, eb_mode, eb, leaf_size, 0, out, out_bytes, perm_out);
}

/* ------------------------------------------------------------------------ */
/* Bit-box reduction (Sec. 4.1, "bit box reduction and bit box intersection */
/* update"; Alg. 1), in rounds.                                              */
/*                                                                          */
/* A bit box is the set of codes a sequence with centre code q_ref and       */
/* widths m can hold: |q_d - q_ref_d| <= 2^(m_d - 1) - 1 on every axis (the  */
/* centre alone when m_d = 0).  Starting from the leaves' boxes (step 4),    */
/* each round selects every alive box whose key (sum of m_d, box index) is   */
/* smaller than the key of every other alive box its box intersects; such    */
/* boxes are pairwise disjoint.  In increasing index, each selected box      */
/* takes from the intersecting alive boxes that are not selected the         */
/* particles inside its bit box (by source box, then position), and becomes  */
/* a sequence: its centre, its remaining own particles in order, then the    */
/* particles it took.  Boxes that lost particles are rebuilt from what they  */
/* keep (step 4 rules) or vanish when empty.  Rounds repeat until no box is  */
/* alive; sequences are written in round order, then box index.  The paper  */
/* removes one box (the smallest sum of m_d) at a time; selecting all local  */
/* minima per round is this implementation's reading, so that rounds run in  */
/* parallel.  one_per_round != 0 selects only the alive box of smallest key  */
/* per round, which is the paper's order (for comparing the two).            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t qref[3], blo[3], bhi[3];
    uint32_t m[3];
    uint32_t key;     /* m_x + m_y + m_z */
    uint64_t centre;  /* particle id */
    int alive;
} rbox;

static int boxes_meet(const rbox *a, const rbox *b)
{
    for (int d = 0; d < 3; d++)
        if (a->blo[d] > b->bhi[d] || b->blo[d] > a->bhi[d]) return 0;
    return 1;
}

static int inside_box(const rbox *b, const int64_t *qp)
{
    for (int d = 0; d < 3; d++)
        if (qp[d] < b->blo[d] || qp[d] > b->bhi[d]) return 0;
    return 1;
}

static int key_less(const rbox *box, uint64_t a, uint64_t b)
{
    if (box[a].key != box[b].key) return box[a].key < box[b].key;
    return a < b;
}

/* Bit box of the live particles ids[0..cnt) (in order), as in step 4. */
static void rebuild_box(const int64_t *q, const uint64_t *ids, const unsigned char *live, uint64_t cnt,
                        int64_t *scratch, uint64_t *slot, rbox *b)
{
    uint64_t k = 0;
    for (uint64_t i = 0; i < cnt; i++)
        if (live[i]) {
            for (int d = 0; d < 3; d++) scratch[3 * k + d] = q[3 * ids[i] + d];
            slot[k++] = i;
        }
    if (k == 0) {
        b->alive = 0;
        return;
    }
    uint64_t c;
    int64_t lo[3], hi[3];
    oracle_bitbox(scratch, k, &c, lo, hi, b->qref, b->m);
    b->centre = ids[slot[c]];
    b->key = b->m[0] + b->m[1] + b->m[2];
    for (int d = 0; d < 3; d++) {
        int64_t h = b->m[d] ? ((1LL << (b->m[d] - 1)) - 1) : 0;
        b->blo[d] = b->qref[d] - h;
        b->bhi[d] = b->qref[d] + h;
    }
    b->alive = 1;
}

int oracle_compress_reduced(const void *pos, uint64_t n, int dtype, int eb_mode, double eb, uint64_t leaf_size,
                            int rule, int one_per_round, uint8_t **out, uint64_t *out_bytes, uint64_t **perm_out,
                            uint64_t *rounds_out)
{
    *out = NULL;
    *out_bytes = 0;
    if (perm_out) *perm_out = NULL;
    if (rounds_out) *rounds_out = 0;
    if (leaf_size < 1) return OR_ERR_ARG;
    oracle_bound b;
    int rc = oracle_error_bound(pos, n, dtype, eb_mode, eb, &b);
    if (rc) return rc;
    if (b.raw) return b.raw_cause; /* the reduction needs codes on every axis */
    int64_t *q = NULL, *scratch = NULL, *sq = NULL;
    uint64_t *order = NULL, *loff = NULL, *lcnt = NULL, *perm = NULL, *slot = NULL, *seq_ids = NULL;
    uint64_t *seq_first = NULL, *seq_wofs = NULL, nl = 0;
    unsigned char *live = NULL, *selected = NULL;
    rbox *box = NULL, *seq_box = NULL;
    uint32_t *words = NULL;
    uint8_t *buf = NULL;
    rc = OR_ERR_NOMEM;
    q = malloc((n ? n : 1) * 3 * sizeof(int64_t));
    order = malloc((n ? n : 1) * sizeof(uint64_t));
    perm = malloc((n ? n : 1) * sizeof(uint64_t));
    live = malloc(n ? n : 1);
    seq_ids = malloc((n ? n : 1) * sizeof(uint64_t));
    if (!q || !order || !perm || !live || !seq_ids) goto done;
    oracle_quantize(pos, n, dtype, &b, q);
    rc = oracle_kdtree_rule(q, n, leaf_size, rule, order, &loff, &lcnt, &nl);
    if (rc) goto done;
    rc = OR_ERR_NOMEM;
    uint64_t maxleaf = 1;
    for (uint64_t L = 0; L < nl; L++)
        if (lcnt[L] > maxleaf) maxleaf = lcnt[L];
    box = calloc(nl ? nl : 1, sizeof(rbox));
    seq_box = calloc(nl ? nl : 1, sizeof(rbox));
    seq_first = malloc((nl + 1) * sizeof(uint64_t));
    seq_wofs = malloc((nl ? nl : 1) * sizeof(uint64_t));
    selected = calloc(nl ? nl : 1, 1);
    scratch = malloc(maxleaf * 3 * sizeof(int64_t));
    sq = malloc(maxleaf * 3 * sizeof(int64_t));
    slot = malloc(maxleaf * sizeof(uint64_t));
    if (!box || !seq_box || !seq_first || !seq_wofs || !selected || !scratch || !sq || !slot) goto done;
    /* initial boxes: the leaves' (live[i] is particle slot i of the leaf order) */
    for (uint64_t i = 0; i < n; i++) live[i] = 1;
    for (uint64_t L = 0; L < nl; L++)
        rebuild_box(q, order + loff[L], live + loff[L], lcnt[L], scratch, slot, &box[L]);

    uint64_t nseq = 0, filled = 0, rounds = 0, alive = nl;
    while (alive) {
        rounds++;
        if (one_per_round) {
            /* the paper's order: only the alive box of smallest key */
            uint64_t best = nl;
            for (uint64_t a = 0; a < nl; a++) {
                selected[a] = 0;
                if (box[a].alive && (best == nl || key_less(box, a, best))) best = a;
            }
            selected[best] = 1;
        } else {
            for (uint64_t a = 0; a < nl; a++) {
                selected[a] = 0;
                if (!box[a].alive) continue;
                int minimal = 1;
                for (uint64_t c = 0; c < nl && minimal; c++)
                    if (c != a && box[c].alive && boxes_meet(&box[a], &box[c]) && key_less(box, c, a)) minimal = 0;
                selected[a] = (unsigned char)minimal;
            }
        }
        for (uint64_t a = 0; a < nl; a++) {
            if (!selected[a]) continue;
            /* the sequence: centre, its own live particles, then what it takes */
            seq_box[nseq] = box[a];
            seq_first[nseq] = filled;
            seq_ids[filled++] = box[a].centre;
            for (uint64_t i = 0; i < lcnt[a]; i++) {
                uint64_t id = order[loff[a] + i];
                if (live[loff[a] + i] && id != box[a].centre) seq_ids[filled++] = id;
                live[loff[a] + i] = 0;
            }
            for (uint64_t c = 0; c < nl; c++) {
                if (c == a || !box[c].alive || selected[c] || !boxes_meet(&box[a], &box[c])) continue;
                int lost = 0;
                for (uint64_t i = 0; i < lcnt[c]; i++) {
                    uint64_t id = order[loff[c] + i];
                    if (live[loff[c] + i] && inside_box(&box[a], &q[3 * id])) {
                        seq_ids[filled++] = id;
                        live[loff[c] + i] = 0;
                        lost = 1;
                    }
                }
                if (lost) box[c].alive = 2; /* to be rebuilt after this round */
            }
            nseq++;
        }
        for (uint64_t a = 0; a < nl; a++) {
            if (selected[a]) box[a].alive = 0;
            if (box[a].alive == 2) rebuild_box(q, order + loff[a], live + loff[a], lcnt[a], scratch, slot, &box[a]);
        }
        alive = 0;
        for (uint64_t a = 0; a < nl; a++) alive += box[a].alive ? 1 : 0;
    }
    seq_first[nseq] = filled;

    /* the stream, as in step 5, with the sequences in place of the leaves */
    uint64_t total_words = 0;
    for (uint64_t k = 0; k < nseq; k++) {
        uint64_t cnt = seq_first[k + 1] - seq_first[k];
        uint64_t bits = (uint64_t)(seq_box[k].m[0] + seq_box[k].m[1] + seq_box[k].m[2]) * (cnt - 1);
        seq_wofs[k] = total_words;
        total_words += (bits + 31) / 32;
    }
    uint64_t bytes = OR_HEADER_BYTES + OR_LEAF_BYTES * nseq + 4 * total_words;
    buf = calloc(bytes, 1);
    words = calloc(total_words ? total_words : 1, sizeof(uint32_t));
    if (!buf || !words) goto done;
    memcpy(buf, "PCB1", 4);
    put_u16(buf + 4, 1);
    buf[6] = (uint8_t)dtype;
    buf[7] = (uint8_t)eb_mode;
    put_u64(buf + 8, n);
    put_f64(buf + 16, eb);
    put_f64(buf + 24, b.eps);
    put_f64(buf + 32, b.s);
    for (int d = 0; d < 3; d++) put_f64(buf + 40 + 8 * d, b.o[d]);
    put_u64(buf + 64, nseq);
    put_u64(buf + 72, total_words);
    put_u32(buf + 80, (uint32_t)leaf_size);
    for (uint64_t k = 0; k < nseq; k++) {
        const rbox *sb = &seq_box[k];
        uint8_t *rec = buf + OR_HEADER_BYTES + OR_LEAF_BYTES * k;
        put_u64(rec + 0, seq_first[k]);
        put_u64(rec + 8, seq_wofs[k]);
        for (int d = 0; d < 3; d++) put_u32(rec + 16 + 4 * d, (uint32_t)(int32_t)sb->qref[d]);
        for (int d = 0; d < 3; d++) rec[28 + d] = (uint8_t)sb->m[d];
        uint64_t bitpos = 32 * seq_wofs[k];
        for (uint64_t i = seq_first[k]; i < seq_first[k + 1]; i++) {
            uint64_t id = seq_ids[i];
            perm[i] = id;
            if (i == seq_first[k]) continue; /* the centre */
            for (int d = 0; d < 3; d++) {
                uint32_t md = sb->m[d];
                if (md == 0) continue;
                int64_t c = (q[3 * id + d] - sb->qref[d]) + ((1LL << (md - 1)) - 1);
                write_bits(words, &bitpos, (uint64_t)c, md);
            }
        }
    }
    for (uint64_t w = 0; w < total_words; w++)
        put_u32(buf + OR_HEADER_BYTES + OR_LEAF_BYTES * nseq + 4 * w, words[w]);
    *out = buf;
    buf = NULL;
    *out_bytes = bytes;
    if (perm_out) {
        *perm_out = perm;
        perm = NULL;
    }
    if (rounds_out) *rounds_out = rounds;
    rc = OR_OK;
done:
    free(q);
    free(order);
    free(loff);
    free(lcnt);
    free(perm);
    free(live);
    free(seq_ids);
    free(box);
    free(seq_box);
    free(seq_first);
    free(seq_wofs);
    free(selected);
    free(scratch);
    free(sq);
    free(slot);
    free(words);
    free(buf);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Reordering for the entropy coder (Sec. 4.2, after Fig. 4): the sequences   */
/* are put in increasing order of sum m_d, and the particles of a sequence    */
/* (its centre staying first) in increasing order of their R-index.  The      */
/* R-index joins a particle's three codes, most significant first, in the     */
/* order of the axes' entropy levels: the entropy of the distribution of m_d  */
/* over all sequences, lowest first (the paper's example: x, then z, then y). */
/* Readings: entropies within 1e-9 of each other tie and keep the x, y, z     */
/* order (a stable insertion sort of the three axes); equal sums of m_d and   */
/* equal R-indices keep the previous order.  Decoding ignores the order, so   */
/* the stream format is unchanged; only positions move.                       */
/* ------------------------------------------------------------------------ */

int oracle_stream_header(const uint8_t *st, uint64_t bytes, uint64_t *n, int *dtype, uint64_t *num_leaves,
                         uint64_t *payload_words);

/* R-index of codes c[3] of widths m[3]: c[order[0]] (highest bits), then
 * c[order[1]], then c[order[2]] (lowest bits); up to 93 bits, as hi:lo. */
void oracle_rindex(const uint32_t c[3], const uint32_t m[3], const int order[3], uint64_t *hi, uint64_t *lo)
{
    uint64_t h = 0, l = 0;
    for (int k = 0; k < 3; k++) {
        uint32_t w = m[order[k]];
        /* (h:l) <<= w, then add the code */
        if (w) {
            if (w >= 64) {
                h = l << (w - 64);
                l = 0;
            } else {
                h = (h << w) | (l >> (64 - w));
                l <<= w;
            }
        }
        l |= (uint64_t)c[order[k]];
    }
    *hi = h;
    *lo = l;
}

/* Axis order by increasing entropy of the m_d distributions of nseq sequences
 * (m is nseq x 3). */
void oracle_axis_order(const uint32_t *m, uint64_t nseq, int order[3], double ent[3])
{
    for (int d = 0; d < 3; d++) {
        uint64_t cnt[32] = {0};
        for (uint64_t k = 0; k < nseq; k++) cnt[m[3 * k + d] & 31]++;
        double h = 0.0;
        for (int v = 0; v < 32; v++)
            if (cnt[v]) {
                double pr = (double)cnt[v] / (double)nseq;
                h -= pr * log2(pr);
            }
        ent[d] = h;
        order[d] = d;
    }
    for (int i = 1; i < 3; i++)
        for (int j = i; j > 0 && ent[order[j]] < ent[order[j - 1]] - 1e-9; j--) {
            int t = order[j];
            order[j] = order[j - 1];
            order[j - 1] = t;
        }
}

typedef struct {
    uint64_t hi, lo, pos; /* R-index, then the particle's place in its sequence */
} rkey;

static int rkey_cmp(const void *a, const void *b)
{
    const rkey *x = a, *y = b;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    return x->pos < y->pos ? -1 : (x->pos > y->pos);
}

typedef struct {
    uint32_t key;
    uint64_t seq;
} skey;

static int skey_cmp(const void *a, const void *b)
{
    const skey *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->seq < y->seq ? -1 : (x->seq > y->seq);
}

int oracle_reorder(const uint8_t *st, uint64_t bytes, const uint64_t *perm_in, uint8_t **out, uint64_t *out_bytes,
                   uint64_t *perm_out, int order_out[3])
{
    *out = NULL;
    *out_bytes = 0;
    uint64_t n, nl, nw;
    int dtype;
    int rc = oracle_stream_header(st, bytes, &n, &dtype, &nl, &nw);
    if (rc) return rc;
    if (st[84]) return OR_ERR_ARG; /* R-indices need codes on every axis */
    const uint8_t *tab = st + OR_HEADER_BYTES;
    const uint8_t *pay = tab + OR_LEAF_BYTES * nl;
    uint32_t *words = malloc((nw ? nw : 1) * sizeof(uint32_t));
    uint32_t *nwords = calloc(nw ? nw : 1, sizeof(uint32_t));
    uint32_t *m = malloc((nl ? nl : 1) * 3 * sizeof(uint32_t));
    uint64_t *po = malloc((nl + 1) * sizeof(uint64_t)), *wo = malloc((nl ? nl : 1) * sizeof(uint64_t));
    skey *sk = malloc((nl ? nl : 1) * sizeof(skey));
    uint32_t *codes = malloc((n ? n : 1) * 3 * sizeof(uint32_t));
    rkey *rk = malloc((n ? n : 1) * sizeof(rkey));
    uint8_t *buf = malloc(bytes);
    rc = OR_ERR_NOMEM;
    if (!words || !nwords || !m || !po || !wo || !sk || !codes || !rk || !buf) goto done;
    for (uint64_t w = 0; w < nw; w++) words[w] = get_u32(pay + 4 * w);
    rc = OR_ERR_CORRUPT;
    for (uint64_t L = 0; L < nl; L++) {
        const uint8_t *rec = tab + OR_LEAF_BYTES * L;
        po[L] = get_u64(rec);
        wo[L] = get_u64(rec + 8);
        for (int d = 0; d < 3; d++) m[3 * L + d] = rec[28 + d];
        if (m[3 * L] > 31 || m[3 * L + 1] > 31 || m[3 * L + 2] > 31) goto done;
    }
    po[nl] = n;
    for (uint64_t L = 0; L < nl; L++) {
        if (po[L + 1] <= po[L]) goto done;
        uint64_t cnt = po[L + 1] - po[L];
        uint64_t need = wo[L] + (((uint64_t)(m[3 * L] + m[3 * L + 1] + m[3 * L + 2]) * (cnt - 1) + 31) / 32);
        if (need > nw) goto done;
        uint64_t bitpos = 32 * wo[L];
        for (uint64_t i = 1; i < cnt; i++)
            for (int d = 0; d < 3; d++) {
                uint32_t md = m[3 * L + d];
                codes[3 * (po[L] + i) + d] = md ? (uint32_t)read_bits(words, bitpos, md) : 0u;
                bitpos += md;
            }
    }
    int order[3];
    double ent[3];
    oracle_axis_order(m, nl, order, ent);
    for (int d = 0; d < 3; d++) order_out[d] = order[d];
    for (uint64_t L = 0; L < nl; L++) {
        sk[L].key = m[3 * L] + m[3 * L + 1] + m[3 * L + 2];
        sk[L].seq = L;
    }
    qsort(sk, nl, sizeof(skey), skey_cmp);
    memcpy(buf, st, OR_HEADER_BYTES);
    uint64_t off = 0, woff = 0;
    for (uint64_t k = 0; k < nl; k++) {
        uint64_t L = sk[k].seq, cnt = po[L + 1] - po[L];
        const uint8_t *rec = tab + OR_LEAF_BYTES * L;
        uint8_t *nrec = buf + OR_HEADER_BYTES + OR_LEAF_BYTES * k;
        memcpy(nrec, rec, OR_LEAF_BYTES);
        put_u64(nrec, off);
        put_u64(nrec + 8, woff);
        /* the centre stays first; the others by R-index, then place */
        for (uint64_t i = 1; i < cnt; i++) {
            oracle_rindex(codes + 3 * (po[L] + i), m + 3 * L, order, &rk[i].hi, &rk[i].lo);
            rk[i].pos = i;
        }
        qsort(rk + 1, cnt - 1, sizeof(rkey), rkey_cmp);
        if (perm_out) perm_out[off] = perm_in ? perm_in[po[L]] : po[L];
        uint64_t bitpos = 32 * woff;
        for (uint64_t i = 1; i < cnt; i++) {
            uint64_t src = po[L] + rk[i].pos;
            if (perm_out) perm_out[off + i] = perm_in ? perm_in[src] : src;
            for (int d = 0; d < 3; d++) {
                uint32_t md = m[3 * L + d];
                if (md) write_bits(nwords, &bitpos, codes[3 * src + d], md);
            }
        }
        off += cnt;
        woff += ((uint64_t)(m[3 * L] + m[3 * L + 1] + m[3 * L + 2]) * (cnt - 1) + 31) / 32;
    }
    for (uint64_t w = 0; w < nw; w++) put_u32(buf + OR_HEADER_BYTES + OR_LEAF_BYTES * nl + 4 * w, nwords[w]);
    *out = buf;
    buf = NULL;
    *out_bytes = bytes;
    rc = OR_OK;
done:
    free(words);
    free(nwords);
    free(m);
    free(po);
    free(wo);
    free(sk);
    free(codes);
    free(rk);
    free(buf);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Step 6: decoding (Sec. 3).  The reconstruction of code q on axis d is     */
/* (T)(o_d + s*q): one double multiply, one double add, one rounding to T.   */
/* ------------------------------------------------------------------------ */

int oracle_stream_header(const uint8_t *st, uint64_t bytes, uint64_t *n, int *dtype, uint64_t *num_leaves,
                         uint64_t *payload_words)
{
    if (bytes < OR_HEADER_BYTES) return OR_ERR_CORRUPT;
    if (memcmp(st, "PCB1", 4) != 0 || get_u16(st + 4) != 1) return OR_ERR_CORRUPT;
    if (st[6] > 1 || st[7] > 1) return OR_ERR_CORRUPT;
    *n = get_u64(st + 8);
    *dtype = st[6];
    *num_leaves = get_u64(st + 64);
    *payload_words = get_u64(st + 72);
    if (*num_leaves > *n) return OR_ERR_CORRUPT;
    if (*num_leaves > (bytes - OR_HEADER_BYTES) / OR_LEAF_BYTES) return OR_ERR_CORRUPT;
    uint64_t rest = bytes - OR_HEADER_BYTES - OR_LEAF_BYTES * *num_leaves;
    if (*payload_words > rest / 4) return OR_ERR_CORRUPT;
    if ((*n > 0) != (*num_leaves > 0)) return OR_ERR_CORRUPT;
    return OR_OK;
}

int oracle_decompress(const uint8_t *st, uint64_t bytes, void *out, uint64_t out_capacity_bytes)
{
    uint64_t n, nl, nw;
    int dtype;
    int rc = oracle_stream_header(st, bytes, &n, &dtype, &nl, &nw);
    if (rc) return rc;
    uint64_t esz = dtype == OR_F32 ? 4 : 8;
    if (out_capacity_bytes < 3 * esz * n) return OR_ERR_CAPACITY;
    double s = get_f64(st + 32), o[3];
    for (int d = 0; d < 3; d++) o[d] = get_f64(st + 40 + 8 * d);
    const uint32_t raw = st[84], M = dtype == OR_F32 ? 32u : 64u;
    if (raw > 7u) return OR_ERR_CORRUPT;
    for (int i = 85; i < 96; i++)
        if (st[i]) return OR_ERR_CORRUPT;
    const uint8_t *tab = st + OR_HEADER_BYTES;
    const uint8_t *pay = tab + OR_LEAF_BYTES * nl;
    uint32_t *words = malloc((nw ? nw : 1) * sizeof(uint32_t));
    if (!words) return OR_ERR_NOMEM;
    for (uint64_t w = 0; w < nw; w++) words[w] = get_u32(pay + 4 * w);
    /* Check every record first, then decode the leaves (each writes its own
     * positions only). */
    uint64_t expect_word = 0;
    rc = OR_OK;
    for (uint64_t L = 0; L < nl; L++) {
        const uint8_t *rec = tab + OR_LEAF_BYTES * L;
        uint64_t po = get_u64(rec), wo = get_u64(rec + 8);
        uint64_t pend = (L + 1 < nl) ? get_u64(rec + OR_LEAF_BYTES) : n;
        uint32_t m[3];
        int bad = 0;
        for (int d = 0; d < 3; d++) {
            m[d] = rec[28 + d];
            bad |= (raw & (1u << d)) ? m[d] != M : m[d] > 31;
        }
        if ((L == 0 && po != 0) || pend <= po || pend > n || wo != expect_word || bad) {
            rc = OR_ERR_CORRUPT;
            break;
        }
        uint64_t bits = (uint64_t)(m[0] + m[1] + m[2]) * (raw ? pend - po : pend - po - 1);
        expect_word = wo + (bits + 31) / 32;
        if (expect_word > nw) {
            rc = OR_ERR_CORRUPT;
            break;
        }
    }
    if (rc == OR_OK) {
#pragma omp parallel for schedule(dynamic, 16)
        for (uint64_t L = 0; L < nl; L++) {
            const uint8_t *rec = tab + OR_LEAF_BYTES * L;
            uint64_t po = get_u64(rec), wo = get_u64(rec + 8);
            uint64_t pend = (L + 1 < nl) ? get_u64(rec + OR_LEAF_BYTES) : n;
            int64_t qref[3];
            uint32_t m[3];
            for (int d = 0; d < 3; d++) {
                qref[d] = (int32_t)get_u32(rec + 16 + 4 * d);
                m[d] = rec[28 + d];
            }
            uint64_t cnt = pend - po;
            uint64_t bitpos = 32 * wo;
            for (uint64_t i = 0; i < cnt; i++) {
                for (int d = 0; d < 3; d++) {
                    if (raw & (1u << d)) { /* the coordinate's own bits */
                        uint64_t u = read_bits(words, bitpos, M);
                        bitpos += M;
                        if (dtype == OR_F32) {
                            uint32_t u32 = (uint32_t)u;
                            memcpy((float *)out + 3 * (po + i) + d, &u32, 4);
                        } else {
                            memcpy((double *)out + 3 * (po + i) + d, &u, 8);
                        }
                        continue;
                    }
                    int64_t qd = qref[d];
                    if ((i > 0 || raw) && m[d] > 0) {
                        uint64_t c = read_bits(words, bitpos, m[d]);
                        bitpos += m[d];
                        qd = qref[d] + (int64_t)c - ((1LL << (m[d] - 1)) - 1);
                    }
                    double y = s * (double)qd;
                    double z = o[d] + y;
                    if (dtype == OR_F32)
                        ((float *)out)[3 * (po + i) + d] = (float)z;
                    else
                        ((double *)out)[3 * (po + i) + d] = z;
                }
            }
        }
    }
    if (rc == OR_OK && expect_word != nw) rc = OR_ERR_CORRUPT;
    free(words);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Step 7: NRMSE and PSNR (Sec. 5.1).  perm maps decoded -> original index.  */
/* ------------------------------------------------------------------------ */

double oracle_nrmse(const void *orig, const void *dec, const uint64_t *perm, uint64_t n, int dtype,
                    double delta_max)
{
    if (n == 0 || !(delta_max > 0.0)) return 0.0;
    double acc = 0.0;
    for (uint64_t i = 0; i < n; i++)
        for (int d = 0; d < 3; d++) {
            double e = (coord(orig, dtype, perm[i], d) - coord(dec, dtype, i, d)) / delta_max;
            acc += e * e;
        }
    return sqrt(acc / (3.0 * (double)n));
}

double oracle_psnr(double nrmse) { return -20.0 * log10(nrmse); }

uint64_t oracle_num_leaves(uint64_t n, uint64_t r) { return r ? leaves_for(n, r) : 0; }

void oracle_free(void *p) { free(p); }
