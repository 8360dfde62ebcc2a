/*
 * oracle.c -- plain CPU oracle for the hierarchical level-of-detail particle renderer
 * of Szalay, Springel & Lemson, "GPU-Based Interactive Visualization of Billion Point
 * Cosmological Simulations" (arXiv:0811.2055).
 *
 * TEST INFRASTRUCTURE ONLY.  The product library never links, loads or calls this file.
 * Only the test-suite, the package smoke check and the benchmark's CPU-baseline leg use
 * it.  It shares no source, header, table or constant generator with the CUDA library;
 * it is written as slow, direct loops so that it can be checked against the paper (and
 * against the readings of the paper listed beside each function) by eye.
 *
 * Build: gcc -O2 -std=gnu11 -ffp-contract=off -fopenmp -fPIC -shared oracle.c -lm
 * (-ffp-contract=off: every float/double operation below rounds on its own; nothing is
 * fused into an FMA.  -fopenmp only splits the points of a frame between threads, each with
 * an image of its own, and the images are summed as integers: the result does not depend on
 * the number of threads; without OpenMP everything runs on one thread.)
 *
 * Precision: FP64 for everything the method does not fix (node geometry, the detail
 * criterion, node masses, statistics); the per-point projection is specified in fp32
 * (one IEEE round-to-nearest per operation) and the per-pixel accumulation in integers,
 * so that a GPU implementation can reproduce the image bit for bit.
 *
 * What pins each function (tests/test_oracle_*.py):
 *   orc_philox4x32_10   published known-answer vectors of Philox4x32-10 (Salmon et al. 2011)
 *   orc_morton_key      octant path obtained by repeated halving of the box (independent)
 *   orc_build           a second, independent construction (orc_build_topdown, recursive
 *                       split by integer coordinate compares, no Morton code); hand-worked
 *                       trees; the invariants fixed by the octree paragraph (at most n points
 *                       per node, children tile the parent, equal mass at every level, every
 *                       particle in exactly one leaf); inclusion statistics of the
 *                       density-weighted subselection; order-freeness under permutation
 *   orc_neglog, orc_cbrt  libm log / cbrt to within 2 ulp
 *   orc_kernel_table    exact high-precision evaluation of the kernel formula
 *   orc_project, orc_splat_*  closed forms: total intensity equals the mass, second moment
 *                       equals 2 sigma^2, centroid on the projected point, mirror symmetry,
 *                       exact shift under a whole-pixel shift of the principal point, and the
 *                       FP64 analytic Gaussian image to within the table-bin bound
 *   orc_render_lod      full-depth render equals the brute-force render of every particle
 *                       (the paper's "indistinguishable from a full rendering" goal at its limit)
 *   orc_select          lambda = 0 gives every visible leaf, lambda = inf gives the root,
 *                       a camera inside a node refines it, depth falls with distance; the
 *                       refine/emit boundary by eyes, lambdas and focal lengths a relative
 *                       1e-9 to either side of hand-worked thresholds (root and child cells,
 *                       on axis, off axis at an edge distance, inside z_near)
 *   orc_tonemap         closed forms on synthetic accumulators
 *   orc_block_quantize  hand-worked codes, the half-step error bound, lossless decode once the
 *                       step is below half an ulp, decode-encode round trips, bounds that
 *                       cover every decoded point, and full depth == brute force of the
 *                       decoded points
 *
 * parity unpinned: which particular n points a node keeps.  The paper fixes only a
 * "density-weighted random subselection"; the generator (Philox4x32-10 keyed on seed,
 * node code and particle id), the exponential-race key and the tie rule are this project's
 * reading.  Given that reading the choice is deterministic, and it is pinned only through
 * the generator's known answers and the inclusion statistics above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_RANGE 2
#define ORC_ERR_OOM 3

#define ORC_LEAF 1
#define ORC_INTERNAL 2
#define ORC_LOSSY 4
#define ORC_REPS 8

#define ORC_MAX_DEPTH 21
#define ORC_T 1024 /* kernel table length */

/* ------------------------------------------------------------------ public structs */

typedef struct {
    double eye[3], right[3], up[3], fwd[3];
    double f_px, cx, cy, z_near;
    int32_t width, height;
} orc_camera;

typedef struct {
    double lambda_px;   /* detail threshold in pixels */
    double sigma_min_px, sigma_max_px;
    double tone_lo, tone_hi; /* fixed tone range (intensity units) when tone_auto == 0 */
    int32_t kernel;     /* 0 Gaussian, 1 cubic spline */
    int32_t tone_auto;
} orc_rparams;

typedef struct {
    uint64_t code, seg_first, point_first, mass_lo, mass_hi;
    uint32_t seg_count, point_count, child_first, child_count;
    int32_t depth, flags, parent, pad;
    float h_cull, w_rep, s_rep, pad2;
    float bmin[3], bmax[3]; /* bounds of the node's particles (cull box before growing) */
} orc_node;

typedef struct {
    orc_node *nodes;
    uint64_t n_nodes;
    float *pts4;      /* stored points: x, y, z, weight */
    float *hs;        /* smoothing length per stored point */
    uint32_t *pt_src; /* sorted position of the particle each stored point copies */
    uint64_t n_pts;
    uint64_t *skey;   /* Morton key per sorted position */
    uint32_t *sidx;   /* input index per sorted position */
    uint64_t n;
    int32_t depth_max;
    int32_t equal_mass;
} orc_tree;

/* ------------------------------------------------------------------ Philox4x32-10 */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
 * ten rounds of two 32x32->64 multiplies, the key bumped by the Weyl constants between
 * rounds. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 64-bit draw for particle `id` inside the node with locational code `code`. */
uint64_t orc_node_draw(uint64_t seed, uint64_t code, uint32_t id)
{
    uint32_t ctr[4] = {id, (uint32_t)code, (uint32_t)(code >> 32), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    return ((uint64_t)r[0] << 32) | (uint64_t)r[1];
}

/* ------------------------------------------------------------------ spec'd series */
/* E(u) = -ln U with U = ((u >> 12) + 1/2) * 2^-52, via the atanh series
 * ln m = 2 atanh((m-1)/(m+1)) = 2 s sum_k s^(2k)/(2k+1), m reduced to [sqrt(1/2), sqrt 2). */
double orc_neglog(uint64_t u)
{
    double U = ((double)(u >> 12) + 0.5) * 0x1p-52;
    int e = 0;
    double m = frexp(U, &e);
    if (m < 0x1.6a09e667f3bcdp-1) {
        m = m * 2.0;
        e = e - 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double p = 1.0 / 25.0;
    for (int k = 11; k >= 0; --k) {
        double t = p * z;
        p = t + 1.0 / (double)(2 * k + 1);
    }
    double lnm = (2.0 * s) * p;
    double lnU = (double)e * 0x1.62e42fefa39efp-1 + lnm;
    return -lnU;
}

/* Cube root of t >= 1 by eight Newton steps s <- (2s + t/s^2)/3 from s0 = 2^ceil(e/3). */
double orc_cbrt(double t)
{
    int e = 0;
    (void)frexp(t, &e);
    int k = e >= 0 ? (e + 2) / 3 : -((-e) / 3);
    double s = ldexp(1.0, k);
    for (int i = 0; i < 8; ++i) {
        double ss = s * s;
        double q = t / ss;
        double num = 2.0 * s + q;
        s = num / 3.0;
    }
    return s;
}

/* ------------------------------------------------------------------ kernel table */
/* Radial kernel sampled at bin centres q_i = (i + 1/2) Qmax / T of q = r^2 / sigma^2, scaled
 * by 2^16 and rounded to the nearest integer.
 *   kernel 0: truncated Gaussian exp(-q/2), Qmax = 9 (support 3 sigma)
 *   kernel 1: M4 cubic spline (Monaghan 1992) with xi = r/h: 1 - 1.5 xi^2 + 0.75 xi^3 (xi < 1),
 *             0.25 (2 - xi)^3 (xi < 2), Qmax = 4 (support 2 h).  The paper's blob is a
 *             "radial cubic function"; the Gaussian is the default workload kernel. */
void orc_kernel_table(int kernel, int32_t *K)
{
    double qmax = kernel == 1 ? 4.0 : 9.0;
    for (int i = 0; i < ORC_T; ++i) {
        double q = ((double)i + 0.5) * qmax / (double)ORC_T;
        double f;
        if (kernel == 1) {
            double xi = sqrt(q);
            if (xi < 1.0) {
                f = 1.0 - 1.5 * q + 0.75 * (q * xi);
            } else {
                double t = 2.0 - xi;
                f = 0.25 * ((t * t) * t);
            }
        } else {
            f = exp(-0.5 * q);
        }
        K[i] = (int32_t)rint(65536.0 * f);
    }
}

/* Normalisations, as fp32 values of the exact expressions (tests check them):
 *   A_gauss = 2^32 / (2 pi (1 - e^-4.5))  (2D Gaussian, renormalised to its 3-sigma disc)
 *   A_cubic = 2^32 * 10 / (7 pi)          (2D M4 spline normalisation, h = 1)
 *   B       = 2^31 / Qmax                 (so that (q S) >> 37 is the table index) */
static const float ORC_A_GAUSS = 0x1.499c68p+29f;
static const float ORC_A_CUBIC = 0x1.d1a452p+30f;
static const float ORC_B_GAUSS = 0x1.c71c72p+27f;
static const float ORC_B_CUBIC = 0x1p+29f;

/* ------------------------------------------------------------------ Morton keys */
/* Root cube [lo, lo + side)^3; per axis q = clamp(floor((x - lo) * 2^21 / side), 0, 2^21-1)
 * in FP64; the key interleaves the bits of (qx, qy, qz) most significant level first with the
 * child octant written as (x << 2) | (y << 1) | z, so bits 62..60 are the level-1 octant. */
static uint32_t orc_quant(float x, double lo, double scale)
{
    double t = ((double)x - lo) * scale;
    if (!(t >= 0.0)) return 0u;
    if (!(t < 2097152.0)) return 2097151u;
    return (uint32_t)t;
}

void orc_quantize(float x, float y, float z, const double lo[3], double side, uint32_t q[3])
{
    double scale = 2097152.0 / side;
    q[0] = orc_quant(x, lo[0], scale);
    q[1] = orc_quant(y, lo[1], scale);
    q[2] = orc_quant(z, lo[2], scale);
}

uint64_t orc_morton_key(float x, float y, float z, const double lo[3], double side)
{
    uint32_t q[3];
    orc_quantize(x, y, z, lo, side, q);
    uint64_t key = 0;
    for (int l = 0; l < ORC_MAX_DEPTH; ++l) {
        int b = ORC_MAX_DEPTH - 1 - l;
        uint64_t o = (uint64_t)(((q[0] >> b) & 1u) << 2 | ((q[1] >> b) & 1u) << 1 | ((q[2] >> b) & 1u));
        key |= o << (60 - 3 * l);
    }
    return key;
}

/* ------------------------------------------------------------------ helpers */
static u128 orc_mass_fixed(float m)
{
    /* m * 2^47 as an exact integer; m in [2^-24, 2^24] has its lowest bit at or above 2^-47. */
    int e = 0;
    double f = frexp((double)m, &e);
    uint64_t mant = (uint64_t)ldexp(f, 24);
    return (u128)mant << (e + 23);
}

static int orc_mass_ok(float m)
{
    return m >= 0x1p-24f && m <= 0x1p+24f;
}

typedef struct {
    uint64_t key;
    uint32_t id;
    uint32_t idx;
} orc_kid;

static int orc_cmp_kid(const void *a, const void *b)
{
    const orc_kid *x = (const orc_kid *)a, *y = (const orc_kid *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

typedef struct {
    double kd;    /* key when masses differ */
    uint64_t ku;  /* key when masses are equal */
    uint32_t id;
    uint32_t pos;
} orc_sel;

static int orc_cmp_sel_u(const void *a, const void *b)
{
    const orc_sel *x = (const orc_sel *)a, *y = (const orc_sel *)b;
    if (x->ku != y->ku) return x->ku < y->ku ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

static int orc_cmp_sel_d(const void *a, const void *b)
{
    const orc_sel *x = (const orc_sel *)a, *y = (const orc_sel *)b;
    if (x->kd != y->kd) return x->kd < y->kd ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

static int orc_cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Density-weighted random subselection of one node (the octree paragraph: a node with more
 * than n points keeps n of them).  Reading: sampling without replacement with inclusion
 * driven by mass -- the exponential race of Efraimidis & Spirakis (2006): keep the n smallest
 * E_i / m_i with E_i = -ln U_i; when every particle has the same mass this is a uniform
 * random n-subset and the raw 64-bit draw itself is the key.  Ties go to the smaller id.
 * `pos` lists the node's particles (sorted positions); on return the first n_sel entries of
 * `chosen` are the kept positions in ascending order. */
void orc_select_node(const uint32_t *pos, const uint32_t *ids, const float *mass, uint64_t count,
                     uint64_t code, uint64_t seed, uint32_t n_sel, int equal_mass, uint32_t *chosen)
{
    orc_sel *s = (orc_sel *)malloc(sizeof(orc_sel) * (count ? count : 1));
    for (uint64_t j = 0; j < count; ++j) {
        uint32_t id = ids[j];
        uint64_t u = orc_node_draw(seed, code, id);
        s[j].ku = u;
        s[j].kd = equal_mass ? 0.0 : orc_neglog(u) / (double)mass[j];
        s[j].id = id;
        s[j].pos = pos[j];
    }
    qsort(s, count, sizeof(orc_sel), equal_mass ? orc_cmp_sel_u : orc_cmp_sel_d);
    for (uint32_t j = 0; j < n_sel; ++j) chosen[j] = s[j].pos;
    qsort(chosen, n_sel, sizeof(uint32_t), orc_cmp_u32);
    free(s);
}

/* ------------------------------------------------------------------ octree build */
/* The octree paragraph: a spatial octree in which every node is represented by at most n
 * points; a node holding more particles is reduced to n by the subselection above, and its
 * children hold the same data at 8x more detail.
 * Readings: a node splits while it holds more than n_max particles and is shallower than
 * depth 21 (the resolution of the 63-bit key); empty octants get no node; a depth-21 node with
 * more than n_max particles is a "lossy leaf" that keeps n_max representatives; leaves keep
 * their particles verbatim; each representative carries the equal weight M_node / n_sel and
 * a smoothing length scaled by cbrt(count / n_sel), the growth of the mean spacing.
 * Nodes are numbered breadth first (depth, then locational code). */
int orc_build(const float *xyz, const float *mass, const float *h, const uint32_t *ids, uint64_t n,
              uint64_t seed, uint32_t n_max, const double lo[3], double side, orc_tree **out)
{
    *out = NULL;
    if (n_max < 1 || !(side > 0.0) || !isfinite(side) || n >= 0xFFFFFFFFull) return ORC_ERR_INVALID;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(lo[a])) return ORC_ERR_INVALID;
    float mmin = 0.0f, mmax = 0.0f;
    for (uint64_t i = 0; i < n; ++i) {
        if (!orc_mass_ok(mass[i])) return ORC_ERR_RANGE;
        if (i == 0 || mass[i] < mmin) mmin = mass[i];
        if (i == 0 || mass[i] > mmax) mmax = mass[i];
    }
    orc_tree *T = (orc_tree *)calloc(1, sizeof(orc_tree));
    T->n = n;
    T->equal_mass = (n == 0) || (mmin == mmax);

    /* keys and the (key, id) order */
    orc_kid *kid = (orc_kid *)malloc(sizeof(orc_kid) * (n ? n : 1));
    for (uint64_t i = 0; i < n; ++i) {
        kid[i].key = orc_morton_key(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lo, side);
        kid[i].id = ids ? ids[i] : (uint32_t)i;
        kid[i].idx = (uint32_t)i;
    }
    qsort(kid, n, sizeof(orc_kid), orc_cmp_kid);
    T->skey = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    T->sidx = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *sid = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    float *smass = (float *)malloc(sizeof(float) * (n ? n : 1));
    for (uint64_t j = 0; j < n; ++j) {
        T->skey[j] = kid[j].key;
        T->sidx[j] = kid[j].idx;
        sid[j] = kid[j].id;
        smass[j] = mass[kid[j].idx];
    }
    free(kid);

    /* breadth-first node list: children are appended in octant order while the list is
     * walked front to back, which yields (depth, code) order */
    uint64_t cap = 64, nn = 0;
    orc_node *N = (orc_node *)calloc(cap, sizeof(orc_node));
    if (n > 0) {
        N[0].code = 1;
        N[0].seg_first = 0;
        N[0].seg_count = (uint32_t)n;
        N[0].depth = 0;
        N[0].parent = -1;
        nn = 1;
    }
    for (uint64_t i = 0; i < nn; ++i) {
        orc_node *nd = &N[i];
        uint64_t b = nd->seg_first, c = nd->seg_count;
        if (c > n_max && nd->depth < ORC_MAX_DEPTH) {
            nd->flags = ORC_INTERNAL | ORC_REPS;
            int sh = 60 - 3 * nd->depth;
            uint64_t j = b;
            nd->child_first = (uint32_t)nn;
            nd->child_count = 0;
            while (j < b + c) {
                uint32_t oct = (uint32_t)((T->skey[j] >> sh) & 7u);
                uint64_t k = j;
                while (k < b + c && (uint32_t)((T->skey[k] >> sh) & 7u) == oct) ++k;
                if (nn == cap) {
                    cap *= 2;
                    N = (orc_node *)realloc(N, cap * sizeof(orc_node));
                    memset(N + nn, 0, (cap - nn) * sizeof(orc_node));
                }
                nd = &N[i];
                N[nn].code = nd->code * 8 + oct;
                N[nn].seg_first = j;
                N[nn].seg_count = (uint32_t)(k - j);
                N[nn].depth = nd->depth + 1;
                N[nn].parent = (int32_t)i;
                nn++;
                nd->child_count++;
                j = k;
            }
        } else if (c > n_max) {
            nd->flags = ORC_LOSSY | ORC_REPS;
        } else {
            nd->flags = ORC_LEAF;
        }
        if (nd->depth > T->depth_max) T->depth_max = nd->depth;
    }

    /* exact node masses */
    for (uint64_t i = 0; i < nn; ++i) {
        u128 M = 0;
        for (uint64_t j = N[i].seg_first; j < N[i].seg_first + N[i].seg_count; ++j) M += orc_mass_fixed(smass[j]);
        N[i].mass_lo = (uint64_t)M;
        N[i].mass_hi = (uint64_t)(M >> 64);
    }

    /* particle bounds per node (NaN coordinates are skipped) */
    for (uint64_t i = 0; i < nn; ++i) {
        for (int a = 0; a < 3; ++a) {
            N[i].bmin[a] = INFINITY;
            N[i].bmax[a] = -INFINITY;
        }
        for (uint64_t j = N[i].seg_first; j < N[i].seg_first + N[i].seg_count; ++j) {
            const float *p = xyz + 3 * (uint64_t)T->sidx[j];
            for (int a = 0; a < 3; ++a) {
                if (p[a] < N[i].bmin[a]) N[i].bmin[a] = p[a];
                if (p[a] > N[i].bmax[a]) N[i].bmax[a] = p[a];
            }
        }
    }

    /* stored points, breadth-first */
    uint64_t np = 0;
    for (uint64_t i = 0; i < nn; ++i) {
        N[i].point_first = np;
        N[i].point_count = (N[i].flags & ORC_REPS) ? n_max : N[i].seg_count;
        np += N[i].point_count;
    }
    T->n_pts = np;
    T->pts4 = (float *)malloc(sizeof(float) * 4 * (np ? np : 1));
    T->hs = (float *)malloc(sizeof(float) * (np ? np : 1));
    T->pt_src = (uint32_t *)malloc(sizeof(uint32_t) * (np ? np : 1));
    for (uint64_t i = 0; i < nn; ++i) {
        orc_node *nd = &N[i];
        uint64_t b = nd->seg_first, c = nd->seg_count, p0 = nd->point_first;
        if (nd->flags & ORC_LEAF) {
            nd->w_rep = 0.0f;
            nd->s_rep = 1.0f;
            for (uint64_t j = 0; j < c; ++j) {
                uint32_t src = T->sidx[b + j];
                T->pts4[4 * (p0 + j) + 0] = xyz[3 * src + 0];
                T->pts4[4 * (p0 + j) + 1] = xyz[3 * src + 1];
                T->pts4[4 * (p0 + j) + 2] = xyz[3 * src + 2];
                T->pts4[4 * (p0 + j) + 3] = mass[src];
                T->hs[p0 + j] = h[src];
                T->pt_src[p0 + j] = (uint32_t)(b + j);
            }
        } else {
            uint32_t *pos = (uint32_t *)malloc(sizeof(uint32_t) * c);
            uint32_t *chosen = (uint32_t *)malloc(sizeof(uint32_t) * c);
            for (uint64_t j = 0; j < c; ++j) pos[j] = (uint32_t)(b + j);
            orc_select_node(pos, sid + b, smass + b, c, nd->code, seed, n_max, T->equal_mass, chosen);
            /* weight: exact mass over n_sel; h scale: cube root of count / n_sel */
            double Md = (double)nd->mass_hi * 18446744073709551616.0 + (double)nd->mass_lo;
            Md = Md * 0x1p-47;
            float w = (float)(Md / (double)n_max);
            double t = (double)c / (double)n_max;
            float s = (float)orc_cbrt(t);
            nd->w_rep = w;
            nd->s_rep = s;
            for (uint32_t j = 0; j < n_max; ++j) {
                uint32_t src = T->sidx[chosen[j]];
                T->pts4[4 * (p0 + j) + 0] = xyz[3 * src + 0];
                T->pts4[4 * (p0 + j) + 1] = xyz[3 * src + 1];
                T->pts4[4 * (p0 + j) + 2] = xyz[3 * src + 2];
                T->pts4[4 * (p0 + j) + 3] = w;
                T->hs[p0 + j] = h[src] * s;
                T->pt_src[p0 + j] = chosen[j];
            }
            free(pos);
            free(chosen);
        }
    }
    /* cull radius: the largest smoothing length drawn anywhere in the subtree */
    for (uint64_t ii = nn; ii-- > 0;) {
        orc_node *nd = &N[ii];
        float hm = 0.0f;
        for (uint64_t j = 0; j < nd->point_count; ++j)
            if (T->hs[nd->point_first + j] > hm) hm = T->hs[nd->point_first + j];
        if (nd->flags & ORC_INTERNAL)
            for (uint32_t k = 0; k < nd->child_count; ++k)
                if (N[nd->child_first + k].h_cull > hm) hm = N[nd->child_first + k].h_cull;
        nd->h_cull = hm;
    }
    free(sid);
    free(smass);
    T->nodes = N;
    T->n_nodes = nn;
    *out = T;
    return ORC_OK;
}

void orc_tree_free(orc_tree *T)
{
    if (!T) return;
    free(T->nodes);
    free(T->pts4);
    free(T->hs);
    free(T->pt_src);
    free(T->skey);
    free(T->sidx);
    free(T);
}

/* ------------------------------------------------------------------ independent construction */
/* Recursive top-down split on integer coordinates (no Morton key): a node at depth d with
 * integer corner (x0, y0, z0) and edge 2^(21-d) sends each particle to the octant given by
 * comparing its quantised coordinates with the midpoint.  Produces the node list (code,
 * depth, count, flags) and each node's member ids; used to cross-check orc_build. */
typedef struct {
    uint64_t code;
    int32_t depth, flags;
    uint32_t count;
    uint32_t *members; /* ids */
} orc_td_node;

typedef struct {
    orc_td_node *v;
    uint64_t n, cap;
} orc_td_list;

static void orc_td_push(orc_td_list *L, orc_td_node nd)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 64;
        L->v = (orc_td_node *)realloc(L->v, L->cap * sizeof(orc_td_node));
    }
    L->v[L->n++] = nd;
}

static void orc_td_rec(orc_td_list *L, const uint32_t (*q)[3], const uint32_t *idv, uint32_t *items, uint64_t cnt,
                       int depth, uint32_t x0, uint32_t y0, uint32_t z0, uint64_t code, uint32_t n_max)
{
    orc_td_node nd;
    nd.code = code;
    nd.depth = depth;
    nd.count = (uint32_t)cnt;
    nd.members = (uint32_t *)malloc(sizeof(uint32_t) * (cnt ? cnt : 1));
    for (uint64_t k = 0; k < cnt; ++k) nd.members[k] = idv[items[k]];
    if (cnt > n_max && depth < ORC_MAX_DEPTH) {
        nd.flags = ORC_INTERNAL | ORC_REPS;
        orc_td_push(L, nd);
        uint32_t half = 1u << (ORC_MAX_DEPTH - 1 - depth);
        for (uint32_t o = 0; o < 8; ++o) {
            uint32_t bx = (o >> 2) & 1u, by = (o >> 1) & 1u, bz = o & 1u;
            uint32_t cx0 = x0 + bx * half, cy0 = y0 + by * half, cz0 = z0 + bz * half;
            uint32_t *sub = (uint32_t *)malloc(sizeof(uint32_t) * (cnt ? cnt : 1));
            uint64_t m = 0;
            for (uint64_t k = 0; k < cnt; ++k) {
                const uint32_t *p = q[items[k]];
                int inx = (p[0] >= x0 + half) == (int)bx;
                int iny = (p[1] >= y0 + half) == (int)by;
                int inz = (p[2] >= z0 + half) == (int)bz;
                if (inx && iny && inz) sub[m++] = items[k];
            }
            if (m > 0) orc_td_rec(L, q, idv, sub, m, depth + 1, cx0, cy0, cz0, code * 8 + o, n_max);
            free(sub);
        }
    } else {
        nd.flags = cnt > n_max ? (ORC_LOSSY | ORC_REPS) : ORC_LEAF;
        orc_td_push(L, nd);
    }
}

static int orc_cmp_td(const void *a, const void *b)
{
    const orc_td_node *x = (const orc_td_node *)a, *y = (const orc_td_node *)b;
    if (x->depth != y->depth) return x->depth < y->depth ? -1 : 1;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    return 0;
}

/* Outputs (caller-allocated, sized by a first call with NULL outputs returning the node count
 * and the total member count through *n_nodes / *n_members): codes, depths, counts, flags in
 * breadth-first order, and the member ids of every node (ascending within a node). */
int orc_build_topdown(const float *xyz, const uint32_t *ids, uint64_t n, uint32_t n_max, const double lo[3],
                      double side, uint64_t *n_nodes, uint64_t *n_members, uint64_t *codes, int32_t *depths,
                      uint32_t *counts, int32_t *flags, uint32_t *members)
{
    uint32_t (*q)[3] = (uint32_t(*)[3])malloc(sizeof(uint32_t[3]) * (n ? n : 1));
    uint32_t *idv = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *items = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint64_t i = 0; i < n; ++i) {
        orc_quantize(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lo, side, q[i]);
        idv[i] = ids ? ids[i] : (uint32_t)i;
        items[i] = (uint32_t)i;
    }
    orc_td_list L = {0, 0, 0};
    if (n > 0) orc_td_rec(&L, (const uint32_t(*)[3])q, idv, items, n, 0, 0, 0, 0, 1, n_max);
    qsort(L.v, L.n, sizeof(orc_td_node), orc_cmp_td);
    uint64_t tot = 0;
    for (uint64_t i = 0; i < L.n; ++i) tot += L.v[i].count;
    *n_nodes = L.n;
    *n_members = tot;
    if (codes) {
        uint64_t off = 0;
        for (uint64_t i = 0; i < L.n; ++i) {
            codes[i] = L.v[i].code;
            depths[i] = L.v[i].depth;
            counts[i] = L.v[i].count;
            flags[i] = L.v[i].flags;
            qsort(L.v[i].members, L.v[i].count, sizeof(uint32_t), orc_cmp_u32);
            memcpy(members + off, L.v[i].members, sizeof(uint32_t) * L.v[i].count);
            off += L.v[i].count;
        }
    }
    for (uint64_t i = 0; i < L.n; ++i) free(L.v[i].members);
    free(L.v);
    free(q);
    free(idv);
    free(items);
    return ORC_OK;
}

/* ------------------------------------------------------------------ projection (fp32 spec) */
/* The per-point work the paper gives to the graphics card ("a smeared blob ... computed for
 * every single pixel of every point").  Reading: a pinhole camera with rows right/up/forward;
 * every operation below is one fp32 IEEE round-to-nearest step, in the order written, with the
 * camera constants rounded to fp32 first; the image y axis points down; positions are
 * quantised to 1/256 pixel and the kernel to a 1024-entry integer table so that the image is
 * an exact integer sum. */
typedef struct {
    float ex, ey, ez, rx, ry, rz, ux, uy, uz, fx, fy, fz;
    float F, CX, CY, ZN, smin, smax, A, B, Rk, Wimg, Himg;
    int32_t row0, row1; /* image rows drawn: [row0, row1) (the whole image unless a window is asked for) */
    int32_t K[ORC_T];
} orc_proj;

typedef struct {
    int32_t U, V; /* position in 1/256 pixel */
    uint32_t S;   /* table scale */
    uint32_t pad;
    uint64_t Wq;  /* amplitude */
} orc_splat;

static void orc_proj_init(orc_proj *P, const orc_camera *c, const orc_rparams *rp)
{
    P->ex = (float)c->eye[0]; P->ey = (float)c->eye[1]; P->ez = (float)c->eye[2];
    P->rx = (float)c->right[0]; P->ry = (float)c->right[1]; P->rz = (float)c->right[2];
    P->ux = (float)c->up[0]; P->uy = (float)c->up[1]; P->uz = (float)c->up[2];
    P->fx = (float)c->fwd[0]; P->fy = (float)c->fwd[1]; P->fz = (float)c->fwd[2];
    P->F = (float)c->f_px;
    P->CX = (float)c->cx;
    P->CY = (float)c->cy;
    P->ZN = (float)c->z_near;
    P->smin = (float)rp->sigma_min_px;
    P->smax = (float)rp->sigma_max_px;
    P->A = rp->kernel == 1 ? ORC_A_CUBIC : ORC_A_GAUSS;
    P->B = rp->kernel == 1 ? ORC_B_CUBIC : ORC_B_GAUSS;
    P->Rk = rp->kernel == 1 ? 2.0f : 3.0f;
    P->Wimg = (float)c->width;
    P->Himg = (float)c->height;
    P->row0 = 0;
    P->row1 = c->height;
    orc_kernel_table(rp->kernel, P->K);
}

/* Returns 1 if the point is drawn (s filled), 0 if culled, -1 if its amplitude is out of
 * the fixed-point range (the point is then not drawn). */
static int orc_project_one(const orc_proj *P, float x, float y, float z, float w, float h, orc_splat *s)
{
    float dx = x - P->ex;
    float dy = y - P->ey;
    float dz = z - P->ez;
    float a, b;
    a = P->rx * dx; b = P->ry * dy; a = a + b; b = P->rz * dz; float xc = a + b;
    a = P->ux * dx; b = P->uy * dy; a = a + b; b = P->uz * dz; float yc = a + b;
    a = P->fx * dx; b = P->fy * dy; a = a + b; b = P->fz * dz; float zc = a + b;
    if (!(zc > P->ZN)) return 0;
    float iz = 1.0f / zc;
    float t = P->F * xc;
    t = t * iz;
    float u = P->CX + t;
    t = P->F * yc;
    t = t * iz;
    float v = P->CY - t;
    float sg = P->F * h;
    sg = sg * iz;
    float sigma = sg >= P->smin ? (sg <= P->smax ? sg : P->smax) : P->smin;
    float s2 = sigma * sigma;
    float wa = w * P->A;
    float Wf = wa / s2;
    float Sf = P->B / s2;
    float R = P->Rk * sigma;
    R = R + 2.0f;
    if (!(u + R >= 0.0f && u - R <= P->Wimg && v + R >= 0.0f && v - R <= P->Himg)) return 0;
    if (!(Wf >= 0.0f && Wf < 0x1p48f)) return -1;
    s->U = (int32_t)lrintf(u * 256.0f);
    s->V = (int32_t)lrintf(v * 256.0f);
    s->Wq = (uint64_t)llrintf(Wf);
    s->S = (uint32_t)llrintf(Sf);
    s->pad = 0;
    return 1;
}

/* exported for the stage tests: out = {drawn, U, V, S, Wq} */
int orc_project(const orc_camera *c, const orc_rparams *rp, float x, float y, float z, float w, float h, int64_t out[5])
{
    orc_proj P;
    orc_proj_init(&P, c, rp);
    orc_splat s;
    int r = orc_project_one(&P, x, y, z, w, h, &s);
    out[0] = r;
    out[1] = r == 1 ? s.U : 0;
    out[2] = r == 1 ? s.V : 0;
    out[3] = r == 1 ? s.S : 0;
    out[4] = r == 1 ? (int64_t)s.Wq : 0;
    return r;
}

/* Adds one splat into the W x H accumulator: every pixel centre (256 px + 128, 256 py + 128)
 * gets floor(Wq K[i] / 2^16) where i = (q S) >> 37 and q is the squared distance in 1/256 px,
 * provided i < 1024.  The pixel loop covers a generous box; the table test decides. */
/* Adds one splat to acc (if acc != NULL) and counts its pixel updates, the (splat, pixel) pairs
 * with a table index below 1024, into *updates (if updates != NULL). */
static void orc_splat_one(const orc_proj *P, const orc_splat *s, int W, int H, uint64_t *acc, uint64_t *updates)
{
    /* support radius in 1/256 px: q S < 1024 * 2^37 needs q < 2^47 / S */
    double qlim = 140737488355328.0 / (double)s->S;
    int64_t r256 = (int64_t)sqrt(qlim) + 256;
    int64_t x0 = ((int64_t)s->U - 128 - r256) / 256 - 1, x1 = ((int64_t)s->U - 128 + r256) / 256 + 1;
    int64_t y0 = ((int64_t)s->V - 128 - r256) / 256 - 1, y1 = ((int64_t)s->V - 128 + r256) / 256 + 1;
    (void)H;
    if (x0 < 0) x0 = 0;
    if (y0 < P->row0) y0 = P->row0;
    if (x1 > W - 1) x1 = W - 1;
    if (y1 > P->row1 - 1) y1 = P->row1 - 1;
    for (int64_t py = y0; py <= y1; ++py) {
        for (int64_t px = x0; px <= x1; ++px) {
            int64_t ddx = px * 256 + 128 - (int64_t)s->U;
            int64_t ddy = py * 256 + 128 - (int64_t)s->V;
            uint64_t q = (uint64_t)(ddx * ddx + ddy * ddy);
            u128 qs = (u128)q * (u128)s->S;
            u128 idx = qs >> 37;
            if (idx < ORC_T) {
                u128 c = ((u128)s->Wq * (u128)(uint32_t)P->K[(int)idx]) >> 16;
                if (acc) acc[(py - P->row0) * W + px] += (uint64_t)c;
                if (updates) ++*updates;
            }
        }
    }
}

/* Threads used by the frame loops below (0: as many as OpenMP offers). */
static int orc_threads = 0;
void orc_set_threads(int n) { orc_threads = n < 0 ? 0 : n; }
int orc_get_threads(void)
{
#ifdef _OPENMP
    return orc_threads > 0 ? orc_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* A list of points to draw: point k is row idx[k] (or row k if idx is NULL) of either float4
 * (x, y, z, weight) rows + h, or of the input layout (xyz rows, mass, h). */
typedef struct {
    const float *pts4, *hs;
    const float *xyz, *mass, *h;
    const uint64_t *idx;
} orc_src;

static void orc_src_get(const orc_src *S, uint64_t k, float *x, float *y, float *z, float *w, float *h)
{
    uint64_t j = S->idx ? S->idx[k] : k;
    if (S->pts4) {
        *x = S->pts4[4 * j]; *y = S->pts4[4 * j + 1]; *z = S->pts4[4 * j + 2]; *w = S->pts4[4 * j + 3];
        *h = S->hs[j];
    } else {
        *x = S->xyz[3 * j]; *y = S->xyz[3 * j + 1]; *z = S->xyz[3 * j + 2]; *w = S->mass[j];
        *h = S->h[j];
    }
}

/* Draws the n points of S into acc (W x H, added to what it holds): R2 then the per-pixel rule
 * of every drawn point.  The points are shared out between threads, each adding into an image of
 * its own; the images are then summed as integers.  Returns ORC_OK, or ORC_ERR_RANGE if a drawn
 * point's amplitude was out of range or the sum of drawn amplitudes reached 2^64 (a pixel could
 * then wrap). */
static int orc_splat_src(const orc_proj *P, const orc_src *S, uint64_t n, int W, int H, uint64_t *acc,
                         uint64_t *n_drawn, uint64_t *n_updates)
{
    int T = orc_get_threads();
    if (T > 64) T = 64;
    (void)H;
    size_t npix = (size_t)W * (size_t)(P->row1 - P->row0);
    uint64_t *img = (uint64_t *)calloc((size_t)T * npix, sizeof(uint64_t));
    int bad[64] = {0};
    u128 tot[64] = {0};
    uint64_t dr[64] = {0}, up[64] = {0};
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(dynamic, 4096)
#endif
    for (uint64_t k = 0; k < n; ++k) {
#ifdef _OPENMP
        int t = omp_get_thread_num();
#else
        int t = 0;
#endif
        float x, y, z, w, h;
        orc_src_get(S, k, &x, &y, &z, &w, &h);
        orc_splat s;
        int r = orc_project_one(P, x, y, z, w, h, &s);
        if (r < 0) bad[t] = 1;
        if (r != 1) continue;
        tot[t] += s.Wq;
        dr[t]++;
        orc_splat_one(P, &s, W, H, img + (size_t)t * npix, n_updates ? &up[t] : NULL);
    }
    int st = ORC_OK;
    u128 total = 0;
    uint64_t drawn = 0, updates = 0;
    for (int t = 0; t < T; ++t) {
        if (bad[t]) st = ORC_ERR_RANGE;
        total += tot[t];
        drawn += dr[t];
        updates += up[t];
    }
    if (n_updates) *n_updates = updates;
    for (size_t i = 0; i < npix; ++i)
        for (int t = 0; t < T; ++t) acc[i] += img[(size_t)t * npix + i];
    free(img);
    if (total >> 64) st = ORC_ERR_RANGE;
    if (n_drawn) *n_drawn = drawn;
    return st;
}

/* Brute-force render of a point list (x, y, z, weight as float4 rows + h): the plain
 * definition of the image.  acc must hold width*height zeros (or a partial image to add to). */
int orc_splat_points(const float *pts4, const float *hs, uint64_t n, const orc_camera *c, const orc_rparams *rp,
                     uint64_t *acc, uint64_t *n_drawn)
{
    orc_proj P;
    orc_proj_init(&P, c, rp);
    orc_src S = {pts4, hs, NULL, NULL, NULL, NULL};
    return orc_splat_src(&P, &S, n, c->width, c->height, acc, n_drawn, NULL);
}

/* Same, from the input layout: xyz rows, mass, h. */
/* Pixel updates of drawing these points: the number of (splat, pixel) pairs inside the support. */
uint64_t orc_count_updates(const float *pts4, const float *hs, uint64_t n, const orc_camera *c, const orc_rparams *rp)
{
    orc_proj P;
    orc_proj_init(&P, c, rp);
    uint64_t updates = 0;
    for (uint64_t i = 0; i < n; ++i) {
        orc_splat s;
        if (orc_project_one(&P, pts4[4 * i], pts4[4 * i + 1], pts4[4 * i + 2], pts4[4 * i + 3], hs[i], &s) != 1)
            continue;
        orc_splat_one(&P, &s, c->width, c->height, NULL, &updates);
    }
    return updates;
}

int orc_splat_particles(const float *xyz, const float *mass, const float *h, uint64_t n, const orc_camera *c,
                        const orc_rparams *rp, uint64_t *acc, uint64_t *n_drawn)
{
    orc_proj P;
    orc_proj_init(&P, c, rp);
    orc_src S = {NULL, NULL, xyz, mass, h, NULL};
    return orc_splat_src(&P, &S, n, c->width, c->height, acc, n_drawn, NULL);
}

/* Image value at one pixel from a point list (for sampled checks of large images). */
uint64_t orc_pixel_value(const float *pts4, const float *hs, uint64_t n, const orc_camera *c, const orc_rparams *rp,
                         int px, int py)
{
    orc_proj P;
    orc_proj_init(&P, c, rp);
    uint64_t acc = 0;
    for (uint64_t i = 0; i < n; ++i) {
        orc_splat s;
        if (orc_project_one(&P, pts4[4 * i], pts4[4 * i + 1], pts4[4 * i + 2], pts4[4 * i + 3], hs[i], &s) != 1)
            continue;
        int64_t ddx = (int64_t)px * 256 + 128 - (int64_t)s.U;
        int64_t ddy = (int64_t)py * 256 + 128 - (int64_t)s.V;
        u128 qs = (u128)(uint64_t)(ddx * ddx + ddy * ddy) * (u128)s.S;
        u128 idx = qs >> 37;
        if (idx < ORC_T) acc += (uint64_t)(((u128)s.Wq * (u128)(uint32_t)P.K[(int)idx]) >> 16);
    }
    return acc;
}

/* ------------------------------------------------------------------ node selection */
/* The paper's view-dependent choice of depth: nodes close to the viewer come from deep in the
 * tree, far ones from shallow levels.  Reading (all FP64):
 *   cull   a node whose particle bounds, grown by Rk * h_cull, lie wholly outside one of five
 *          half-spaces:
 *          z >= z_near, and the four planes through the eye and the image borders moved out
 *          by M = Rk * sigma_min + 2 pixels (so no point whose clamped blob reaches the image
 *          is lost);
 *   refine an internal node iff (f * edge)^2 > lambda^2 * max(D^2, z_near^2), D the distance
 *          from the eye to the node's box (0 inside): its n representatives would each cover
 *          more than about one pixel at lambda = sqrt(n);
 *   emit   every other visible node (its stored points are drawn). */
typedef struct {
    double n[5][3];
    double off[5];
    double E[3];
    double F, lam, zn, rk;
} orc_frustum;

static void orc_frustum_init(orc_frustum *Fr, const orc_camera *c, const orc_rparams *rp)
{
    double rk = rp->kernel == 1 ? 2.0 : 3.0;
    double M = rk * rp->sigma_min_px + 2.0;
    double F = c->f_px;
    double cl = c->cx + M;
    double cr = ((double)c->width + M) - c->cx;
    double ct = c->cy + M;
    double cb = ((double)c->height + M) - c->cy;
    for (int a = 0; a < 3; ++a) {
        Fr->n[0][a] = c->fwd[a];
        Fr->n[1][a] = F * c->right[a] + cl * c->fwd[a];
        Fr->n[2][a] = -(F * c->right[a]) + cr * c->fwd[a];
        Fr->n[3][a] = -(F * c->up[a]) + ct * c->fwd[a];
        Fr->n[4][a] = F * c->up[a] + cb * c->fwd[a];
        Fr->E[a] = c->eye[a];
    }
    Fr->off[0] = -c->z_near;
    Fr->off[1] = Fr->off[2] = Fr->off[3] = Fr->off[4] = 0.0;
    Fr->F = F;
    Fr->lam = rp->lambda_px;
    Fr->zn = c->z_near;
    Fr->rk = rk;
}

static void orc_node_box(const orc_node *nd, const double lo[3], double side, double blo[3], double bhi[3], double *edge)
{
    int d = nd->depth;
    uint64_t p = nd->code ^ ((uint64_t)1 << (3 * d));
    uint32_t q[3] = {0, 0, 0};
    for (int l = 0; l < d; ++l) {
        uint32_t o = (uint32_t)((p >> (3 * (d - 1 - l))) & 7u);
        q[0] = (q[0] << 1) | ((o >> 2) & 1u);
        q[1] = (q[1] << 1) | ((o >> 1) & 1u);
        q[2] = (q[2] << 1) | (o & 1u);
    }
    double e = ldexp(side, -d);
    for (int a = 0; a < 3; ++a) {
        blo[a] = lo[a] + e * (double)q[a];
        bhi[a] = blo[a] + e;
    }
    *edge = e;
}

/* 1 = culled, 2 = refine, 3 = emit */
static int orc_classify(const orc_frustum *Fr, const orc_node *nd, const double lo[3], double side)
{
    double blo[3], bhi[3], e;
    orc_node_box(nd, lo, side, blo, bhi, &e);
    double rho = Fr->rk * (double)nd->h_cull;
    for (int k = 0; k < 5; ++k) {
        double s = Fr->off[k];
        for (int a = 0; a < 3; ++a) {
            double na = Fr->n[k][a];
            double pa = na > 0.0 ? ((double)nd->bmax[a] + rho) - Fr->E[a] : ((double)nd->bmin[a] - rho) - Fr->E[a];
            s = s + na * pa;
        }
        if (s < 0.0) return 1;
    }
    if (!(nd->flags & ORC_INTERNAL)) return 3;
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double da = Fr->E[a] < blo[a] ? blo[a] - Fr->E[a] : (Fr->E[a] > bhi[a] ? Fr->E[a] - bhi[a] : 0.0);
        d2 = d2 + da * da;
    }
    double fe = Fr->F * e;
    double lhs = fe * fe;
    double zn2 = Fr->zn * Fr->zn;
    double rhs = (Fr->lam * Fr->lam) * (d2 > zn2 ? d2 : zn2);
    return lhs > rhs ? 2 : 3;
}

/* Emits node indices (any order) into out (capacity n_nodes); returns how many. */
int64_t orc_select(const orc_tree *T, const double lo[3], double side, const orc_camera *c, const orc_rparams *rp,
                   uint32_t *out)
{
    if (T->n_nodes == 0) return 0;
    orc_frustum Fr;
    orc_frustum_init(&Fr, c, rp);
    uint32_t *stack = (uint32_t *)malloc(sizeof(uint32_t) * (T->n_nodes + 1));
    int64_t sp = 0, m = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        uint32_t i = stack[--sp];
        const orc_node *nd = &T->nodes[i];
        int k = orc_classify(&Fr, nd, lo, side);
        if (k == 1) continue;
        if (k == 3) {
            out[m++] = i;
            continue;
        }
        for (uint32_t j = nd->child_count; j-- > 0;) stack[sp++] = nd->child_first + j;
    }
    free(stack);
    return m;
}

/* LOD render: the brute-force image of exactly the points stored in the selected nodes. */
/* Draws the points stored in the nodes sel[0..m) (rows [row0, row1) of the image; acc holds
 * width * (row1 - row0) values). */
static int orc_render_nodes(const orc_tree *T, const uint32_t *sel, int64_t m, const orc_camera *c,
                            const orc_rparams *rp, int32_t row0, int32_t row1, uint64_t *acc, uint64_t *n_drawn,
                            uint64_t *n_points, uint64_t *n_updates)
{
    if (row0 < 0) row0 = 0;
    if (row1 > c->height) row1 = c->height;
    if (row1 < row0) row1 = row0;
    uint64_t np = 0;
    for (int64_t k = 0; k < m; ++k) np += T->nodes[sel[k]].point_count;
    uint64_t *rows = (uint64_t *)malloc(sizeof(uint64_t) * (np + 1));
    uint64_t q = 0;
    for (int64_t k = 0; k < m; ++k) {
        const orc_node *nd = &T->nodes[sel[k]];
        for (uint64_t j = nd->point_first; j < nd->point_first + nd->point_count; ++j) rows[q++] = j;
    }
    orc_proj P;
    orc_proj_init(&P, c, rp);
    P.row0 = row0;
    P.row1 = row1;
    orc_src S = {T->pts4, T->hs, NULL, NULL, NULL, rows};
    int st = orc_splat_src(&P, &S, np, c->width, c->height, acc, n_drawn, n_updates);
    free(rows);
    if (n_points) *n_points = np;
    return st;
}

/* Rows [row0, row1) of the LOD frame (acc holds width * (row1 - row0) values): the same
 * selection, projection and per-pixel rule as the whole frame, with the pixel loops limited to
 * those rows, so the result is exactly those rows of the whole frame. */
int orc_render_lod_rows(const orc_tree *T, const double lo[3], double side, const orc_camera *c,
                        const orc_rparams *rp, int32_t row0, int32_t row1, uint64_t *acc, uint64_t *n_drawn,
                        uint64_t *n_points, uint64_t *n_updates)
{
    uint32_t *sel = (uint32_t *)malloc(sizeof(uint32_t) * (T->n_nodes + 1));
    int64_t m = orc_select(T, lo, side, c, rp, sel);
    int st = orc_render_nodes(T, sel, m, c, rp, row0, row1, acc, n_drawn, n_points, n_updates);
    free(sel);
    return st;
}

/* Part `part` of `n_parts` of a split frame: of the nodes the frame selects, only those whose index
 * in the node table is congruent to `part` modulo `n_parts` are drawn.  Summing the parts' images
 * as integers gives the whole frame (each selected node is drawn by exactly one part). */
int orc_render_lod_part(const orc_tree *T, const double lo[3], double side, const orc_camera *c,
                        const orc_rparams *rp, int32_t part, int32_t n_parts, uint64_t *acc, uint64_t *n_drawn,
                        uint64_t *n_points)
{
    uint32_t *sel = (uint32_t *)malloc(sizeof(uint32_t) * (T->n_nodes + 1));
    int64_t m = orc_select(T, lo, side, c, rp, sel), k = 0;
    for (int64_t j = 0; j < m; ++j)
        if (n_parts <= 1 || (int64_t)(sel[j] % (uint32_t)n_parts) == part) sel[k++] = sel[j];
    int st = orc_render_nodes(T, sel, k, c, rp, 0, c->height, acc, n_drawn, n_points, NULL);
    free(sel);
    return st;
}

/* The whole frame, with its pixel-update count. */
int orc_render_lod_counted(const orc_tree *T, const double lo[3], double side, const orc_camera *c,
                           const orc_rparams *rp, uint64_t *acc, uint64_t *n_drawn, uint64_t *n_points,
                           uint64_t *n_updates)
{
    return orc_render_lod_rows(T, lo, side, c, rp, 0, c->height, acc, n_drawn, n_points, n_updates);
}

/* The whole frame. */
int orc_render_lod(const orc_tree *T, const double lo[3], double side, const orc_camera *c, const orc_rparams *rp,
                   uint64_t *acc, uint64_t *n_drawn, uint64_t *n_points)
{
    return orc_render_lod_rows(T, lo, side, c, rp, 0, c->height, acc, n_drawn, n_points, NULL);
}

/* Overwrites the points stored in node `node` with `count` (= its point_count) new ones:
 * pts4 (x, y, z, weight per point) and hs.  The node's particle bounds and h_cull, and those of
 * every ancestor, grow to cover the new points (each coordinate or h enters as v + 0, so -0
 * counts as +0), so that culling stays conservative for what is drawn; the points copy no
 * particle any more (pt_src = 0xFFFFFFFF).  Returns ORC_OK or ORC_ERR_INVALID. */
int orc_tree_set_points(orc_tree *T, uint32_t node, const float *pts4, const float *hs, uint64_t count)
{
    if (node >= T->n_nodes || count != T->nodes[node].point_count) return ORC_ERR_INVALID;
    uint64_t pf = T->nodes[node].point_first;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, hm = -INFINITY;
    for (uint64_t i = 0; i < count; ++i) {
        for (int a = 0; a < 4; ++a) T->pts4[4 * (pf + i) + a] = pts4[4 * i + a];
        T->hs[pf + i] = hs[i];
        if (T->pt_src) T->pt_src[pf + i] = 0xFFFFFFFFu;
        for (int a = 0; a < 3; ++a) {
            float v = pts4[4 * i + a] + 0.0f;
            if (v < mn[a]) mn[a] = v;
            if (v > mx[a]) mx[a] = v;
        }
        float h = hs[i] + 0.0f;
        if (h > hm) hm = h;
    }
    if (count == 0) return ORC_OK;
    for (int32_t k = (int32_t)node; k >= 0; k = T->nodes[k].parent) {
        orc_node *nd = &T->nodes[k];
        for (int a = 0; a < 3; ++a) {
            if (mn[a] < nd->bmin[a]) nd->bmin[a] = mn[a];
            if (mx[a] > nd->bmax[a]) nd->bmax[a] = mx[a];
        }
        if (hm > nd->h_cull) nd->h_cull = hm;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ 16-bit block codes */
/* Storage paragraph: every point's position is kept as 2 bytes per coordinate spanning the
 * block (node) that holds it, and the other properties are coded the same way.  Readings:
 *   position  per node: qlo[a] = fp32(corner of the node's cell), qstep = fp32(edge 2^-16);
 *             code = floor(((double)x - qlo) / qstep) clamped to [0, 65535] (NaN -> 0);
 *             decode x' = qlo + (code + 1/2) qstep, fp32, one rounding per operation.  A point
 *             inside its cell comes back within edge 2^-17 (plus the final fp32 rounding);
 *             once qstep is below half an fp32 ulp of x the decode returns x itself.
 *   w and h   per node: lo = the smallest finite value, step = fp32((largest - lo) / 65535)
 *             in double; code = rne(((double)v - lo) / step) clamped to [0, 65535] (0 when
 *             step is 0 or v is not finite); decode v' = lo + code step, fp32.
 *   culling   the quantised tree's node bounds and h_cull are recomputed from the decoded
 *             points of each subtree, so culling stays conservative for what is drawn. */
static uint16_t orc_code_floor(float x, float lo, float step)
{
    double d = ((double)x - (double)lo) / (double)step;
    if (!(d >= 0.0)) return 0;
    if (d >= 65535.0) return 65535;
    return (uint16_t)floor(d);
}

static uint16_t orc_code_rne(float v, float lo, float step)
{
    if (!(step > 0.0f) || !isfinite(v)) return 0;
    double d = rint(((double)v - (double)lo) / (double)step);
    if (!(d >= 0.0)) return 0;
    if (d >= 65535.0) return 65535;
    return (uint16_t)d;
}

static float orc_decode_pos(uint16_t c, float lo, float step)
{
    float t = (float)c + 0.5f;
    float m = t * step;
    return lo + m;
}

static float orc_decode_lin(uint16_t c, float lo, float step)
{
    float m = (float)c * step;
    return lo + m;
}

static void orc_range(const float *v, uint64_t n, uint64_t stride, float *lo, float *step)
{
    float mn = 0.0f, mx = 0.0f;
    int any = 0;
    for (uint64_t j = 0; j < n; ++j) {
        float x = v[j * stride];
        if (!isfinite(x)) continue;
        if (!any || x < mn) mn = x;
        if (!any || x > mx) mx = x;
        any = 1;
    }
    *lo = mn + 0.0f; /* a zero lower bound is stored as +0 whichever zero came first */
    *step = (float)(((double)mx - (double)mn) / 65535.0);
}

/* Encodes every stored point of T.  codes: 5 per point (x, y, z, w, h); qa: 8 floats per node
 * (qlo x, y, z, qstep, w lo, w step, h lo, h step).  *decoded receives a tree with the same
 * nodes whose points are the decoded values and whose bmin / bmax / h_cull cover the decoded
 * points of each subtree (pt_src, skey, sidx are not carried over). */
int orc_block_quantize(const orc_tree *T, const double lo[3], double side, uint16_t *codes, float *qa,
                       orc_tree **decoded)
{
    uint64_t nn = T->n_nodes, np = T->n_pts;
    orc_tree *D = (orc_tree *)calloc(1, sizeof(orc_tree));
    D->nodes = (orc_node *)malloc(sizeof(orc_node) * (nn ? nn : 1));
    D->pts4 = (float *)malloc(sizeof(float) * 4 * (np ? np : 1));
    D->hs = (float *)malloc(sizeof(float) * (np ? np : 1));
    D->n_nodes = nn;
    D->n_pts = np;
    D->n = T->n;
    D->depth_max = T->depth_max;
    D->equal_mass = T->equal_mass;
    if (nn) memcpy(D->nodes, T->nodes, sizeof(orc_node) * nn);
    for (uint64_t i = 0; i < nn; ++i) {
        const orc_node *nd = &T->nodes[i];
        double blo[3], bhi[3], e;
        orc_node_box(nd, lo, side, blo, bhi, &e);
        float *A = qa + 8 * i;
        for (int a = 0; a < 3; ++a) A[a] = (float)blo[a];
        A[3] = (float)ldexp(e, -16);
        uint64_t p0 = nd->point_first, m = nd->point_count;
        orc_range(T->pts4 + 4 * p0 + 3, m, 4, &A[4], &A[5]);
        orc_range(T->hs + p0, m, 1, &A[6], &A[7]);
        for (uint64_t j = p0; j < p0 + m; ++j) {
            uint16_t *c = codes + 5 * j;
            for (int a = 0; a < 3; ++a) c[a] = orc_code_floor(T->pts4[4 * j + a], A[a], A[3]);
            c[3] = orc_code_rne(T->pts4[4 * j + 3], A[4], A[5]);
            c[4] = orc_code_rne(T->hs[j], A[6], A[7]);
            for (int a = 0; a < 3; ++a) D->pts4[4 * j + a] = orc_decode_pos(c[a], A[a], A[3]);
            D->pts4[4 * j + 3] = orc_decode_lin(c[3], A[4], A[5]);
            D->hs[j] = orc_decode_lin(c[4], A[6], A[7]);
        }
    }
    /* subtree bounds and h_cull of the decoded points, children before parents */
    for (uint64_t ii = nn; ii-- > 0;) {
        orc_node *nd = &D->nodes[ii];
        float mn[3], mx[3], hm = 0.0f;
        for (int a = 0; a < 3; ++a) {
            mn[a] = INFINITY;
            mx[a] = -INFINITY;
        }
        for (uint64_t j = nd->point_first; j < nd->point_first + nd->point_count; ++j) {
            for (int a = 0; a < 3; ++a) {
                float x = D->pts4[4 * j + a];
                if (x < mn[a]) mn[a] = x;
                if (x > mx[a]) mx[a] = x;
            }
            if (D->hs[j] > hm) hm = D->hs[j];
        }
        if (nd->flags & ORC_INTERNAL)
            for (uint32_t k = 0; k < nd->child_count; ++k) {
                const orc_node *ch = &D->nodes[nd->child_first + k];
                for (int a = 0; a < 3; ++a) {
                    if (ch->bmin[a] < mn[a]) mn[a] = ch->bmin[a];
                    if (ch->bmax[a] > mx[a]) mx[a] = ch->bmax[a];
                }
                if (ch->h_cull > hm) hm = ch->h_cull;
            }
        for (int a = 0; a < 3; ++a) {
            nd->bmin[a] = mn[a];
            nd->bmax[a] = mx[a];
        }
        nd->h_cull = hm;
    }
    *decoded = D;
    return ORC_OK;
}

/* single-value helpers for the tests */
void orc_block_code_pos(const float *x, uint64_t n, float lo, float step, uint16_t *out)
{
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_code_floor(x[i], lo, step);
}

void orc_block_decode_pos(const uint16_t *c, uint64_t n, float lo, float step, float *out)
{
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_decode_pos(c[i], lo, step);
}

void orc_block_code_lin(const float *v, uint64_t n, float lo, float step, uint16_t *out)
{
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_code_rne(v[i], lo, step);
}

void orc_block_decode_lin(const uint16_t *c, uint64_t n, float lo, float step, float *out)
{
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_decode_lin(c[i], lo, step);
}

/* ------------------------------------------------------------------ tone map */
/* Log scale to 8-bit grey (the paper shows density renders without giving the map).
 * Reading: I = acc * 2^-32; out = 0 if I <= lo, else min(255, rne(255 ln(I/lo) / ln(hi/lo)));
 * automatic range: hi = the largest I in the image, lo = 1e-4 hi. */
void orc_tonemap(const uint64_t *acc, uint64_t npix, const orc_rparams *rp, uint8_t *out)
{
    double hi, lo;
    if (rp->tone_auto) {
        uint64_t mx = 0;
        for (uint64_t i = 0; i < npix; ++i)
            if (acc[i] > mx) mx = acc[i];
        hi = ldexp((double)mx, -32);
        lo = hi * 1e-4;
    } else {
        hi = rp->tone_hi;
        lo = rp->tone_lo;
    }
    if (!(hi > 0.0) || !(lo > 0.0) || !(hi > lo)) {
        memset(out, 0, npix);
        return;
    }
    double den = log(hi / lo);
    for (uint64_t i = 0; i < npix; ++i) {
        double I = ldexp((double)acc[i], -32);
        if (I <= lo) {
            out[i] = 0;
            continue;
        }
        double t = rint(255.0 * log(I / lo) / den);
        out[i] = (uint8_t)(t > 255.0 ? 255.0 : t);
    }
}

/* ------------------------------------------------------------------ batch helpers */
void orc_morton_keys(const float *xyz, uint64_t n, const double lo[3], double side, uint64_t *out)
{
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_morton_key(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lo, side);
}

void orc_node_draws(uint64_t seed, uint64_t code, const uint32_t *ids, uint64_t n, uint64_t *out)
{
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_node_draw(seed, code, ids[i]);
}

void orc_neglogs(const uint64_t *u, uint64_t n, double *out)
{
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_neglog(u[i]);
}

/* fp32 normalisation constants, for the tests: {A_gauss, A_cubic, B_gauss, B_cubic} */
void orc_constants(float out[4])
{
    out[0] = ORC_A_GAUSS;
    out[1] = ORC_A_CUBIC;
    out[2] = ORC_B_GAUSS;
    out[3] = ORC_B_CUBIC;
}
