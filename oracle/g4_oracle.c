/*
 * g4_oracle.c -- plain, slow, FP64 CPU reference for the short-range tree/FMM gravity path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is checked against.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * Every function follows the definition or the algorithm steps of GADGET-4 (Springel et al.
 * 2021) in the paper's order and notation, with no blocking, fusion or reordering beyond
 * what that definition states:
 *   - integer coordinates ................ Sec. 2.10 "Integer coordinates", Sec. 2.11
 *   - Peano-Hilbert keys / oct-tree ....... Sec. 2.2.1 "Geometry of the tree"
 *   - multipole moments Q_n ............... Sec. 2.2.2, definition below Eq. (eqonesidetreepotential)
 *   - derivative tensors D_n, g_n ......... Eqs. (eqngderiv0)-(eqngderiv), Appendix A
 *   - softening law ....................... Eq. (eqnsoft), Sec. 2.1
 *   - TreePM short-range kernel ........... Eq. (eqnpo4), Sec. 2.3
 *   - one-sided walk, opening criteria .... Eqs. (eqonesidetreepotential), (eqonesidetreeacc),
 *                                           (eqnrelcriterion), Sec. 2.2.3
 *   - FMM expansion, dual walk, L2L/L2P ... Sec. 2.4 and Appendix A
 *
 * Readings of places where the paper is silent are listed in the header of each function.
 * Parity pins (tests/test_oracle_*.py) tie each function to closed forms, invariants and
 * brute force, independent of this code.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXP 5
#define OR_KEYBITS 21

typedef struct {
    double box;        /* L: the integer unit is L / 2^32 */
    int periodic;      /* 1: nearest periodic image (Sec. 2.1, Eq. eqnpo1) */
    double r_s;        /* TreePM split scale; <= 0 means plain Newtonian kernel */
    double r_cut;      /* absolute short-range cutoff radius (Sec. 2.3); ignored when r_s <= 0 */
    int pp_cut;        /* 1: particle pairs at r >= r_cut are dropped */
    double alpha;      /* relative opening parameter, Eq. (eqnrelcriterion) */
    double theta;      /* geometric opening angle theta_c */
    int criterion;     /* 0 = relative, 1 = geometric */
    int order;         /* expansion order p (1..5) */
    int exclusion;     /* 1: exclusion zone around node centres (Sec. 2.2.3) */
    double G;          /* gravitational constant */
    int n_eps;         /* number of softening classes */
    const double *eps; /* softening length eps_0 per class (Sec. 2.7) */
    int keep_qp;       /* FMM: 1 keeps Q_p in the potential (Sec. 2.4 drops it by default) */
    int soft_nodes;    /* tree walk and FMM: 0 opens every pair closer than 2.8 max(eps)
                          (GADGET-3); 1 applies the GADGET-4 rule of Sec. 2.7 (softened
                          multipoles) */
    int ewald;         /* tree walk, periodic and r_s = 0: 1 adds the Ewald correction psi to
                          every interaction (Sec. 2.2.4, Eqs. eqnpo1, eqnewal) */
} or_params;

/* ===================================================================================== */
/* a1: integer coordinates (Sec. 2.10, Sec. 2.11)                                         */
/* ===================================================================================== */

/* Periodic box: x_int = floor(x / L * 2^32) mod 2^32.  Out is SoA 3 x n. */
void or_int_coords_periodic(const double *pos, int64_t n, double L, uint32_t *out)
{
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) {
            double t = floor(pos[3 * i + k] / L * 4294967296.0);
            int64_t v = (int64_t)t;
            out[k * n + i] = (uint32_t)(v & 0xFFFFFFFFLL);
        }
}

/* Isolated system (Sec. 2.11): the particles are shrink-wrapped and mapped into the central
 * half of the integer cube, so that integer differences never wrap.  Reading: cube side S is
 * the smallest power of two >= 2 * (largest bounding-box extent); the cube is centred on the
 * bounding-box midpoint.  frame = {origin_x, origin_y, origin_z, S}, with physical position =
 * origin + x_int * S / 2^32. */
void or_int_coords_isolated(const double *pos, int64_t n, uint32_t *out, double *frame)
{
    double lo[3], hi[3], c[3];
    for (int k = 0; k < 3; k++) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) {
            double x = pos[3 * i + k];
            if (x < lo[k]) lo[k] = x;
            if (x > hi[k]) hi[k] = x;
        }
    double ext = 0.0;
    for (int k = 0; k < 3; k++) {
        c[k] = 0.5 * (lo[k] + hi[k]);
        if (hi[k] - lo[k] > ext) ext = hi[k] - lo[k];
    }
    /* smallest power of two S with S >= 2 * ext (S = 1 for a single point) */
    double S = 1.0;
    if (ext > 0.0) {
        int e;
        double f = frexp(2.0 * ext, &e);   /* 2*ext = f * 2^e, f in [0.5, 1) */
        S = (f == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
    }
    double scale = 4294967296.0 / S;
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) {
            double t = floor((pos[3 * i + k] - c[k]) * scale) + 2147483648.0;
            out[k * n + i] = (uint32_t)(int64_t)t;
        }
    for (int k = 0; k < 3; k++) frame[k] = c[k] - 0.5 * S;
    frame[3] = S;
}

/* ===================================================================================== */
/* a2: Peano-Hilbert key (Sec. 2.2.1; curve construction after Skilling 2004,             */
/*     "Programming the Hilbert curve", restated here in plain C)                         */
/* ===================================================================================== */

/* Key of the cell (x, y, z), each given with `bits` bits.  The three coordinates are first
 * turned into the "transposed" Hilbert index: walking from the most significant bit down, a
 * set bit at level q inverts the lower bits of the first axis, a clear bit swaps the lower
 * bits of the first axis with those of the current axis; afterwards the axes are Gray-coded.
 * The key interleaves the transposed bits, x first, most significant level first. */
uint64_t or_hilbert_key(uint32_t x, uint32_t y, uint32_t z, int bits)
{
    uint32_t X[3] = {x, y, z};
    uint32_t top = 1u << (bits - 1);
    for (uint32_t q = top; q > 1; q >>= 1) {
        uint32_t low = q - 1;
        for (int ax = 0; ax < 3; ax++) {
            if (X[ax] & q) {
                X[0] ^= low;
            } else {
                uint32_t t = (X[0] ^ X[ax]) & low;
                X[0] ^= t;
                X[ax] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t flip = 0;
    for (uint32_t q = top; q > 1; q >>= 1)
        if (X[2] & q) flip ^= q - 1;
    for (int ax = 0; ax < 3; ax++) X[ax] ^= flip;
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; b--)
        for (int ax = 0; ax < 3; ax++)
            key = (key << 1) | ((X[ax] >> b) & 1u);
    return key;
}

/* 63-bit key from the top 21 bits of each 32-bit coordinate. */
void or_keys(const uint32_t *pos, int64_t n, uint64_t *keys)
{
    for (int64_t i = 0; i < n; i++)
        keys[i] = or_hilbert_key(pos[i] >> 11, pos[n + i] >> 11, pos[2 * n + i] >> 11,
                                 OR_KEYBITS);
}

/* a3: stable sort of (key, original index); perm[sorted] = original index. */
typedef struct { uint64_t key; int64_t idx; } or_kv;
static int or_kv_cmp(const void *a, const void *b)
{
    const or_kv *p = (const or_kv *)a, *q = (const or_kv *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx ? 1 : 0);
}

void or_sort(const uint64_t *keys, int64_t n, uint64_t *keys_sorted, int64_t *perm)
{
    or_kv *a = (or_kv *)malloc(sizeof(or_kv) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) { a[i].key = keys[i]; a[i].idx = i; }
    qsort(a, (size_t)n, sizeof(or_kv), or_kv_cmp);
    for (int64_t i = 0; i < n; i++) { keys_sorted[i] = a[i].key; perm[i] = a[i].idx; }
    free(a);
}

/* ===================================================================================== */
/* a4: oct-tree with a leaf threshold (Sec. 2.2.1)                                        */
/* ===================================================================================== */

typedef struct {
    int64_t nn, cap;
    int32_t *level;
    int64_t *first, *count, *next;  /* next = index after the node's subtree (DFS pre-order) */
    uint32_t *center;               /* nn x 3 geometric centre in integer units */
    /* filled by or_multipoles */
    int order;
    double *mass;                   /* nn */
    double *com;                    /* nn x 3: (s - c) in physical units */
    double *mono;                   /* nn x nmono: monomial moments of orders 0..order */
    double *eps_max, *amin;         /* nn */
    double *eps_min;                /* nn: smallest softening among the node's particles */
} or_tree;

static int64_t or_nmono(int order) { return (int64_t)(order + 1) * (order + 2) * (order + 3) / 6; }

/* offset of multi-index (a, b, c), a + b + c = n, within all monomials of orders 0..n */
static int or_mono_index(int a, int b, int c)
{
    int n = a + b + c;
    return n * (n + 1) * (n + 2) / 6 + (n - a) * (n - a + 1) / 2 + (n - a - b);
}

static void or_tree_push(or_tree *t, int level, int64_t first, int64_t count,
                         const uint32_t *pos, int64_t np)
{
    if (t->nn == t->cap) {
        t->cap = t->cap * 2 + 64;
        t->level = (int32_t *)realloc(t->level, sizeof(int32_t) * t->cap);
        t->first = (int64_t *)realloc(t->first, sizeof(int64_t) * t->cap);
        t->count = (int64_t *)realloc(t->count, sizeof(int64_t) * t->cap);
        t->next = (int64_t *)realloc(t->next, sizeof(int64_t) * t->cap);
        t->center = (uint32_t *)realloc(t->center, sizeof(uint32_t) * 3 * t->cap);
    }
    int64_t k = t->nn++;
    t->level[k] = level;
    t->first[k] = first;
    t->count[k] = count;
    t->next[k] = -1;
    /* the cell of a level-l node is the common top-l-bit prefix of its particles' coordinates */
    for (int ax = 0; ax < 3; ax++) {
        uint32_t x = pos[ax * np + first];
        uint32_t corner = (level == 0) ? 0u : (x & ~((1u << (32 - level)) - 1u));
        uint32_t half = (level == 0) ? 0x80000000u : (1u << (31 - level));
        t->center[3 * k + ax] = corner + half;
    }
}

/* Recursive subdivision in depth-first pre-order, children in PH order.  A node is split
 * when it holds more than leaf_max particles and has not reached the key resolution. */
static void or_build_rec(or_tree *t, const uint64_t *keys, const uint32_t *pos, int64_t np,
                         int level, int64_t first, int64_t count, int leaf_max)
{
    int64_t me = t->nn;
    or_tree_push(t, level, first, count, pos, np);
    if (count > leaf_max && level < OR_KEYBITS) {
        int shift = 3 * (OR_KEYBITS - level - 1);
        int64_t i = first, end = first + count;
        while (i < end) {
            uint64_t digit = (keys[i] >> shift) & 7u;
            int64_t j = i;
            while (j < end && ((keys[j] >> shift) & 7u) == digit) j++;
            or_build_rec(t, keys, pos, np, level + 1, i, j - i, leaf_max);
            i = j;
        }
    }
    t->next[me] = t->nn;
}

or_tree *or_tree_build(const uint64_t *keys_sorted, const uint32_t *pos_sorted, int64_t n,
                       int leaf_max)
{
    or_tree *t = (or_tree *)calloc(1, sizeof(or_tree));
    if (n > 0) or_build_rec(t, keys_sorted, pos_sorted, n, 0, 0, n, leaf_max);
    return t;
}

int64_t or_tree_nnodes(const or_tree *t) { return t->nn; }

void or_tree_export(const or_tree *t, int32_t *level, int64_t *first, int64_t *count,
                    int64_t *next, uint32_t *center)
{
    memcpy(level, t->level, sizeof(int32_t) * t->nn);
    memcpy(first, t->first, sizeof(int64_t) * t->nn);
    memcpy(count, t->count, sizeof(int64_t) * t->nn);
    memcpy(next, t->next, sizeof(int64_t) * t->nn);
    memcpy(center, t->center, sizeof(uint32_t) * 3 * t->nn);
}

void or_tree_free(or_tree *t)
{
    if (!t) return;
    free(t->level); free(t->first); free(t->count); free(t->next); free(t->center);
    free(t->mass); free(t->com); free(t->mono); free(t->eps_max); free(t->amin); free(t->eps_min);
    free(t);
}

/* ===================================================================================== */
/* a5: node moments by definition (Sec. 2.2.2): M, centre of mass s, and                  */
/*     Q_n = sum_j m_j (x_j - s)^(n), stored as monomials sum m dx^a dy^b dz^c.            */
/* ===================================================================================== */

static double or_isep(uint32_t a, uint32_t b, int periodic)
{
    /* signed integer difference a - b: two's complement gives the nearest image (Sec. 2.10) */
    if (periodic) return (double)(int32_t)(a - b);
    return (double)((int64_t)a - (int64_t)b);
}

static double or_ipow(double x, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; i++) r *= x;
    return r;
}

void or_multipoles(or_tree *t, const uint32_t *pos, int64_t np, const double *mass,
                   const uint8_t *cls, const double *aold, const or_params *P)
{
    int order = P->order;
    int64_t nm = or_nmono(order);
    double scale = P->box / 4294967296.0;
    t->order = order;
    t->mass = (double *)realloc(t->mass, sizeof(double) * (t->nn ? t->nn : 1));
    t->com = (double *)realloc(t->com, sizeof(double) * 3 * (t->nn ? t->nn : 1));
    t->mono = (double *)realloc(t->mono, sizeof(double) * nm * (t->nn ? t->nn : 1));
    t->eps_max = (double *)realloc(t->eps_max, sizeof(double) * (t->nn ? t->nn : 1));
    t->eps_min = (double *)realloc(t->eps_min, sizeof(double) * (t->nn ? t->nn : 1));
    t->amin = (double *)realloc(t->amin, sizeof(double) * (t->nn ? t->nn : 1));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < t->nn; k++) {
        int64_t f = t->first[k], e = f + t->count[k];
        double M = 0.0, d[3] = {0, 0, 0}, em = 0.0, am = INFINITY, en = INFINITY;
        for (int64_t j = f; j < e; j++) {
            M += mass[j];
            for (int ax = 0; ax < 3; ax++)
                d[ax] += mass[j] * or_isep(pos[ax * np + j], t->center[3 * k + ax], 0) * scale;
            double ej = P->eps[cls ? cls[j] : 0];
            if (ej > em) em = ej;
            if (ej < en) en = ej;
            double aj = aold ? aold[j] : 0.0;
            if (aj < am) am = aj;
        }
        double s[3];
        for (int ax = 0; ax < 3; ax++) s[ax] = (M > 0) ? d[ax] / M : 0.0;
        t->mass[k] = M;
        for (int ax = 0; ax < 3; ax++) t->com[3 * k + ax] = s[ax];
        t->eps_max[k] = em;
        t->eps_min[k] = en;
        t->amin[k] = am;
        double *q = t->mono + nm * k;
        for (int64_t c = 0; c < nm; c++) q[c] = 0.0;
        for (int64_t j = f; j < e; j++) {
            double dx[3];
            for (int ax = 0; ax < 3; ax++)
                dx[ax] = or_isep(pos[ax * np + j], t->center[3 * k + ax], 0) * scale - s[ax];
            for (int n = 0; n <= order; n++)
                for (int a = n; a >= 0; a--)
                    for (int b = n - a; b >= 0; b--) {
                        int c = n - a - b;
                        q[or_mono_index(a, b, c)] +=
                            mass[j] * or_ipow(dx[0], a) * or_ipow(dx[1], b) * or_ipow(dx[2], c);
                    }
        }
    }
}

void or_tree_export_moments(const or_tree *t, double *mass, double *com, double *mono,
                            double *eps_max, double *amin)
{
    int64_t nm = or_nmono(t->order);
    memcpy(mass, t->mass, sizeof(double) * t->nn);
    memcpy(com, t->com, sizeof(double) * 3 * t->nn);
    memcpy(mono, t->mono, sizeof(double) * nm * t->nn);
    if (eps_max) memcpy(eps_max, t->eps_max, sizeof(double) * t->nn);
    if (amin) memcpy(amin, t->amin, sizeof(double) * t->nn);
}

/* ===================================================================================== */
/* a7: interaction kernels                                                                 */
/* ===================================================================================== */

/* Cubic-spline softened inverse distance g_soft(r) = 1/(r + eps(r)) = -W_2(u)/h with
 * h = 2.8 eps_0, u = r/h (Eq. eqnsoft).  W_2 is the potential of the cubic spline kernel
 * (Springel et al. 2001, eq. 71, not printed in the paper; reading: the standard form).
 * Returns g0 = g_soft and g1 = (1/r) d g_soft / dr. */
void or_soft_kernel(double r, double h, double *g0, double *g1)
{
    if (r >= h) {
        *g0 = 1.0 / r;
        *g1 = -1.0 / (r * r * r);
        return;
    }
    double u = r / h, u2 = u * u;
    double W, dWu; /* W_2(u) and W_2'(u)/u */
    if (u < 0.5) {
        W = 16.0 / 3.0 * u2 - 48.0 / 5.0 * u2 * u2 + 32.0 / 5.0 * u2 * u2 * u - 14.0 / 5.0;
        dWu = 32.0 / 3.0 - 192.0 / 5.0 * u2 + 32.0 * u2 * u;
    } else {
        W = 1.0 / (15.0 * u) + 32.0 / 3.0 * u2 - 16.0 * u2 * u + 48.0 / 5.0 * u2 * u2
            - 32.0 / 15.0 * u2 * u2 * u - 16.0 / 5.0;
        dWu = -1.0 / (15.0 * u2 * u) + 64.0 / 3.0 - 48.0 * u + 192.0 / 5.0 * u2
              - 32.0 / 3.0 * u2 * u;
    }
    *g0 = -W / h;
    *g1 = -dWu / (h * h * h);
}

/* Pair kernel of the short-range potential, Eq. (eqnpo4):
 *   g(r) = g_soft(r) - 1/r + erfc(r / 2 r_s) / r = g_soft(r) - erf(r / 2 r_s) / r
 * (the constant pi/(alpha^2 V) is dropped, as in Sec. 2.3).  Plain Newtonian softened kernel
 * when r_s <= 0.  g1 = g'(r)/r.  h = 2.8 eps_ij with eps_ij = max(eps_i, eps_j). */
void or_pair_kernel(double r, double h, double r_s, double *g0, double *g1)
{
    or_soft_kernel(r, h, g0, g1);
    if (r_s <= 0.0) return;
    double al = 0.5 / r_s, x = al * r;
    const double tsp = 1.1283791670955126; /* 2/sqrt(pi) */
    if (x < 1e-3) {
        /* series of erf(x)/x and of its r-derivative term near the origin */
        *g0 -= al * tsp * (1.0 - x * x / 3.0 + x * x * x * x / 10.0);
        *g1 += al * al * al * tsp * (2.0 / 3.0 - 0.4 * x * x + x * x * x * x / 7.0);
        return;
    }
    double ef = erf(x);
    *g0 -= ef / r;
    /* -(1/r) d/dr [erf(al r)/r] = erf(al r)/r^3 - (2 al/sqrt(pi)) exp(-al^2 r^2) / r^2 */
    *g1 += ef / (r * r * r) - al * tsp * exp(-x * x) / (r * r);
}

/* g_n(r) = (r^-1 d/dr)^n g(r) for n = 0..nmax (Eq. above eqngderiv0), for the unsoftened
 * multipole kernel g = 1/r (r_s <= 0) or g = erfc(r / 2 r_s) / r.  The ordinary derivatives
 * g^(k) come from Leibniz' rule on erfc(al r) * (1/r) with
 *   d^j/dr^j erfc(al r) = -(2 al / sqrt(pi)) (-al)^(j-1) H_{j-1}(al r) exp(-al^2 r^2),
 * H the physicists' Hermite polynomials; g_n then follows from the Appendix A formulas. */
void or_gn(double r, double r_s, int nmax, double *g)
{
    double E[8], R[8], gd[8];
    int kmax = nmax;
    if (r_s > 0.0) {
        double al = 0.5 / r_s, x = al * r, ex = exp(-x * x);
        double H[8];
        H[0] = 1.0;
        H[1] = 2.0 * x;
        for (int m = 1; m < 7; m++) H[m + 1] = 2.0 * x * H[m] - 2.0 * m * H[m - 1];
        E[0] = erfc(x);
        double alp = 1.0; /* (-al)^(j-1) */
        for (int j = 1; j <= kmax; j++) {
            E[j] = -1.1283791670955126 * al * alp * H[j - 1] * ex;
            alp *= -al;
        }
    } else {
        E[0] = 1.0;
        for (int j = 1; j <= kmax; j++) E[j] = 0.0;
    }
    double fact = 1.0, rp = 1.0 / r;
    for (int i = 0; i <= kmax; i++) {
        R[i] = ((i & 1) ? -1.0 : 1.0) * fact * rp; /* d^i/dr^i (1/r) = (-1)^i i! / r^(i+1) */
        fact *= (double)(i + 1);
        rp /= r;
    }
    for (int k = 0; k <= kmax; k++) {
        double s = 0.0, binom = 1.0;
        for (int j = 0; j <= k; j++) {
            s += binom * E[j] * R[k - j];
            binom = binom * (double)(k - j) / (double)(j + 1);
        }
        gd[k] = s;
    }
    /* Appendix A: g_n = r^-n sum_j c_{n,j} g^(n-j) / r^j */
    static const double C[8][7] = {
        {0},
        {1},
        {1, -1},
        {1, -3, 3},
        {1, -6, 15, -15},
        {1, -10, 45, -105, 105},
        {1, -15, 105, -420, 945, -945},
        {1, -21, 210, -1260, 4725, -10395, 10395},
    };
    g[0] = gd[0];
    for (int n = 1; n <= nmax; n++) {
        double s = 0.0, rj = 1.0;
        for (int j = 0; j < n; j++) {
            s += C[n][j] * gd[n - j] * rj;
            rj /= r;
        }
        g[n] = s * or_ipow(1.0 / r, n);
    }
}

/* g_n = (r^-1 d/dr)^n g for the softened kernel used by softened multipoles (Sec. 2.7):
 * g = g_soft(r) for r_s <= 0, g = g_soft(r) - erf(r / 2 r_s) / r for TreePM, with
 * g_soft = -W_2(u) / h (u = r / h < 1; W_2 the cubic-spline potential of or_soft_kernel) and
 * 1/r beyond h.  On a piece W_2 = sum_k c_k u^k (k = -1, 0, 2, 3, 4, 5) the operator
 * r^-1 d/dr maps u^k to (k / h^2) u^(k-2), so
 *   g_n = -(1/h) sum_k c_k [k (k-2) ... (k-2n+2)] u^(k-2n) / h^(2n);
 * the TreePM part is -erf/r = erfc/r - 1/r, i.e. or_gn with r_s minus or_gn without. */
void or_gn_soft(double r, double h, double r_s, int nmax, double *g)
{
    if (r >= h) { or_gn(r, r_s, nmax, g); return; }
    static const int kk[6] = {-1, 0, 2, 3, 4, 5};
    const double c_in[6] = {0.0, -14.0 / 5.0, 16.0 / 3.0, 0.0, -48.0 / 5.0, 32.0 / 5.0};
    const double c_out[6] = {1.0 / 15.0, -16.0 / 5.0, 32.0 / 3.0, -16.0, 48.0 / 5.0, -32.0 / 15.0};
    const double *c = (r / h < 0.5) ? c_in : c_out;
    double u = r / h;
    for (int n = 0; n <= nmax; n++) {
        double sum = 0.0;
        for (int t = 0; t < 6; t++) {
            if (c[t] == 0.0) continue;
            double f = 1.0;
            for (int m = 0; m < n; m++) f *= (double)(kk[t] - 2 * m);
            if (f == 0.0) continue;
            sum += c[t] * f * pow(u, (double)(kk[t] - 2 * n));
        }
        g[n] = -sum / h / pow(h, 2.0 * n);
    }
    if (r_s > 0.0) {
        double ge[OR_MAXP + 2], gN[OR_MAXP + 2];
        or_gn(r, r_s, nmax, ge);
        or_gn(r, 0.0, nmax, gN);
        for (int n = 0; n <= nmax; n++) g[n] += ge[n] - gN[n];
    }
}

/* Full derivative tensor D_m = grad^(m) g(|r|) (3^m entries, index digit k of the flat index
 * is the k-th tensor index, little-endian in base 3).  Eqs. (eqngderiv0)-(eqngderiv): each
 * component is a sum over all partial pairings of its m index slots; a pairing with j pairs
 * contributes g_{m-j} times one Kronecker delta per pair and one r component per unpaired
 * slot. */
static double or_pairings(int m, const int *idx, const double *r, const double *g,
                          unsigned used, double prod, int pairs)
{
    int k = 0;
    while (k < m && (used & (1u << k))) k++;
    if (k == m) return g[m - pairs] * prod;
    used |= 1u << k;
    double s = or_pairings(m, idx, r, g, used, prod * r[idx[k]], pairs);
    for (int v = k + 1; v < m; v++)
        if (!(used & (1u << v)) && idx[v] == idx[k])
            s += or_pairings(m, idx, r, g, used | (1u << v), prod, pairs + 1);
    return s;
}

static int or_pow3(int m)
{
    int p = 1;
    for (int i = 0; i < m; i++) p *= 3;
    return p;
}

void or_D_full(int m, const double *r, const double *g, double *out)
{
    int n3 = or_pow3(m), idx[16];
    for (int t = 0; t < n3; t++) {
        int v = t;
        for (int k = 0; k < m; k++) { idx[k] = v % 3; v /= 3; }
        out[t] = or_pairings(m, idx, r, g, 0u, 1.0, 0);
    }
}

/* full-tensor component of a symmetric moment tensor: the monomial of its index counts */
static double or_Q_full(const double *mono, int m, int t)
{
    int cnt[3] = {0, 0, 0};
    for (int k = 0; k < m; k++) { cnt[t % 3]++; t /= 3; }
    return mono[or_mono_index(cnt[0], cnt[1], cnt[2])];
}

static double or_factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; i++) f *= i;
    return f;
}

/* ===================================================================================== */
/* a6: one-sided tree walk (Sec. 2.2.2-2.2.3, Sec. 2.3)                                   */
/* ===================================================================================== */

/* Particle-node term with r = s - x:
 *   phi += -G sum_{n=0}^{p}   (1/n!) Q_n . D_n        (Eq. eqonesidetreepotential)
 *   a   += -G sum_{n=0}^{p-1} (1/n!) Q_n . D_{n+1}    (Eq. eqonesidetreeacc)            */
static void or_pn_h(const double *mono, const double *rv, int p, double r_s, double h, double G,
                    double *acc, double *pot)
{
    double r = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
    double g[OR_MAXP + 2];
    if (h > 0.0) or_gn_soft(r, h, r_s, p, g);
    else or_gn(r, r_s, p, g);
    double D[OR_MAXP + 1][729];
    for (int m = 0; m <= p; m++) or_D_full(m, rv, g, D[m]);
    double phi = 0.0, a[3] = {0, 0, 0};
    for (int n = 0; n <= p; n++) {
        double inv = 1.0 / or_factorial(n);
        int n3 = or_pow3(n);
        for (int t = 0; t < n3; t++) {
            double q = or_Q_full(mono, n, t);
            phi += inv * q * D[n][t];
            if (n <= p - 1)
                for (int i = 0; i < 3; i++) a[i] += inv * q * D[n + 1][i + 3 * t];
        }
    }
    *pot += -G * phi;
    for (int i = 0; i < 3; i++) acc[i] += -G * a[i];
}

/* the unsoftened particle-node term */
static void or_pn(const double *mono, const double *rv, int p, double r_s, double G,
                  double *acc, double *pot)
{
    or_pn_h(mono, rv, p, r_s, 0.0, G, acc, pot);
}

static double or_sep(uint32_t a, uint32_t b, const or_params *P)
{
    return or_isep(a, b, P->periodic) * (P->box / 4294967296.0);
}

/* Ewald correction tensors (defined with the Ewald sums below) */
#define OR_EW_MMAX (OR_MAXP + 1)
void or_ewald_dpsi(const double *x, double L, int mmax, double (*D)[729]);
double or_ewald_psi(const double *x, double L, double alpha, int nr, int nk);

/* Ewald correction of an accepted node (pure periodic tree, Sec. 2.2.4): the correction
 * potential psi of Eq. (eqnpo1) expanded about the node's centre of mass like the Newtonian
 * term, with r = s - x (nearest image):
 *   phi += +G sum_{n=0}^{p}   (1/n!) Q_n . D_n[psi](r)
 *   a   += +G sum_{n=0}^{p-1} (1/n!) Q_n . D_{n+1}[psi](r)                                */
static void or_pn_ewald(const double *mono, const double *rv, int p, double L, double G,
                        double *acc, double *pot)
{
    static __thread double D[OR_EW_MMAX + 1][729];
    or_ewald_dpsi(rv, L, p, D);
    double phi = 0.0, a[3] = {0, 0, 0};
    for (int n = 0; n <= p; n++) {
        double inv = 1.0 / or_factorial(n);
        int n3 = or_pow3(n);
        for (int t = 0; t < n3; t++) {
            double q = or_Q_full(mono, n, t);
            phi += inv * q * D[n][t];
            if (n <= p - 1)
                for (int i = 0; i < 3; i++) a[i] += inv * q * D[n + 1][i + 3 * t];
        }
    }
    *pot += G * phi;
    for (int i = 0; i < 3; i++) acc[i] += G * a[i];
}

/* Ewald correction of one particle pair, d = x_j - x (nearest image): m psi(d), m grad psi(d) */
static void or_pp_ewald(const double *d, double m, double L, double G, double *acc, double *pot)
{
    static __thread double D[OR_EW_MMAX + 1][729];
    or_ewald_dpsi(d, L, 1, D);
    *pot += G * m * D[0][0];
    for (int i = 0; i < 3; i++) acc[i] += G * m * D[1][i];
}

/* Walk for the particle at sorted index i.  Node handling, in this order:
 *   - TreePM: the node is dropped when the nearest point of its (nearest-image) cube is
 *     further than r_cut (Sec. 2.3, reading: Euclidean distance to the cube);
 *   - a leaf is opened into particle-particle terms (pairs at r >= r_cut are dropped when
 *     pp_cut is set);
 *   - an internal node is opened if the particle lies inside the node's cube, or inside the
 *     exclusion cube of half-width l around the geometric centre (Sec. 2.2.3, reading of
 *     Fig. FigTREESketch), or if r < 2.8 max(eps_i, eps_max(node)) and either the
 *     GADGET-3 rule is in force (multipoles always unsoftened) or, under the GADGET-4 rule of
 *     Sec. 2.7, both eps_i and the node's smallest softening lie below eps_ij (otherwise the
 *     multipole of the softened kernel with eps_ij is used), or if the criterion fails:
 *       relative  G M / r^2 (l / r)^p < alpha |a_old|     (Eq. eqnrelcriterion)
 *       geometric l / r < theta_c;
 *     otherwise its multipole expansion is used.                                          */
static void or_walk_one(const or_tree *t, const uint32_t *pos, int64_t np, const double *mass,
                        const uint8_t *cls, const double *aold, int64_t i, const or_params *P,
                        double *acc, double *pot, int64_t *cnt)
{
    double scale = P->box / 4294967296.0;
    int p = P->order;
    int64_t nm = or_nmono(p);
    int treepm = P->r_s > 0.0;
    double rc2 = P->r_cut * P->r_cut;
    double eps_i = P->eps[cls ? cls[i] : 0];
    double a_i = aold ? aold[i] : 0.0;
    uint32_t xi[3] = {pos[i], pos[np + i], pos[2 * np + i]};
    acc[0] = acc[1] = acc[2] = 0.0;
    *pot = 0.0;
    cnt[0] = cnt[1] = 0;
    const int ewald = P->ewald && P->periodic && !treepm;
    if (ewald) {   /* the particle's own periodic images: m_i psi(0) (no force) */
        const double z[3] = {0.0, 0.0, 0.0};
        *pot += P->G * mass[i] * or_ewald_psi(z, P->box, 2.0 / P->box, 2, 5);
    }
    int64_t k = 0;
    while (k < t->nn) {
        double side = ldexp(P->box, -t->level[k]);
        double dc[3];
        for (int ax = 0; ax < 3; ax++) dc[ax] = or_sep(t->center[3 * k + ax], xi[ax], P);
        if (treepm) {
            double e2 = 0.0;
            for (int ax = 0; ax < 3; ax++) {
                double e = fabs(dc[ax]) - 0.5 * side;
                if (e > 0) e2 += e * e;
            }
            if (e2 > rc2) { k = t->next[k]; continue; }
        }
        int leaf = (t->next[k] == k + 1);
        if (leaf) {
            for (int64_t j = t->first[k]; j < t->first[k] + t->count[k]; j++) {
                if (j == i) continue;
                double d[3];
                for (int ax = 0; ax < 3; ax++) d[ax] = or_sep(pos[ax * np + j], xi[ax], P);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (treepm && P->pp_cut && r2 >= rc2) continue;
                double eps_j = P->eps[cls ? cls[j] : 0];
                double h = 2.8 * (eps_i > eps_j ? eps_i : eps_j);
                double g0, g1;
                or_pair_kernel(sqrt(r2), h, P->r_s, &g0, &g1);
                *pot += -P->G * mass[j] * g0;
                for (int ax = 0; ax < 3; ax++) acc[ax] += -P->G * mass[j] * g1 * d[ax];
                if (ewald) or_pp_ewald(d, mass[j], P->box, P->G, acc, pot);
                cnt[0]++;
            }
            k = t->next[k];
            continue;
        }
        double rv[3];
        for (int ax = 0; ax < 3; ax++) rv[ax] = dc[ax] + t->com[3 * k + ax];
        double r2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
        double dmax = fmax(fabs(dc[0]), fmax(fabs(dc[1]), fabs(dc[2])));
        int open = 0;
        if (dmax <= 0.5 * side) open = 1;                     /* particle inside the node */
        if (P->exclusion && dmax < side) open = 1;             /* exclusion zone */
        double epsn = t->eps_max[k];
        double h = 2.8 * (eps_i > epsn ? eps_i : epsn);        /* 2.8 eps_ij */
        int softened = r2 < h * h;
        if (softened) {
            if (!P->soft_nodes) open = 1;                      /* GADGET-3: always open */
            /* GADGET-4 (Sec. 2.7): open only if both the particle's and the node's smallest
             * softening are below eps_ij (a mixed node some of whose pairs would be
             * oversoftened); otherwise use the multipole of the softened kernel */
            else if (2.8 * eps_i < h && 2.8 * t->eps_min[k] < h) open = 1;
        }
        if (!open) {
            if (P->criterion == 1) {
                if (side * side >= P->theta * P->theta * r2) open = 1;
            } else {
                double r = sqrt(r2);
                double lhs = P->G * t->mass[k] * or_ipow(side, p);
                double rhs = P->alpha * a_i * or_ipow(r, p + 2);
                if (!(lhs < rhs)) open = 1;
            }
        }
        if (open) { k = k + 1; continue; }
        or_pn_h(t->mono + nm * k, rv, p, P->r_s, softened ? h : 0.0, P->G, acc, pot);
        if (ewald) or_pn_ewald(t->mono + nm * k, rv, p, P->box, P->G, acc, pot);
        cnt[1]++;
        k = t->next[k];
    }
}

void or_tree_walk(const or_tree *t, const uint32_t *pos, int64_t np, const double *mass,
                  const uint8_t *cls, const double *aold, const int64_t *sinks, int64_t ns,
                  const or_params *P, double *acc, double *pot, int64_t *cnt)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < ns; s++)
        or_walk_one(t, pos, np, mass, cls, aold, sinks[s], P, acc + 3 * s, pot + s, cnt + 2 * s);
}

/* ===================================================================================== */
/* Direct summation (validation reference, Sec. 3): every pair, nearest periodic image.   */
/* r_max > 0 restricts the sum to pairs with r < r_max (cell list when periodic).          */
/* ===================================================================================== */

static void or_pair_acc(const uint32_t *pos, int64_t np, const double *mass, const uint8_t *cls,
                        int64_t i, int64_t j, const or_params *P, double *acc, double *pot,
                        double r2max)
{
    double d[3];
    for (int ax = 0; ax < 3; ax++) d[ax] = or_sep(pos[ax * np + j], pos[ax * np + i], P);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2max > 0 && r2 >= r2max) return;
    double ei = P->eps[cls ? cls[i] : 0], ej = P->eps[cls ? cls[j] : 0];
    double h = 2.8 * (ei > ej ? ei : ej), g0, g1;
    or_pair_kernel(sqrt(r2), h, P->r_s, &g0, &g1);
    *pot += -P->G * mass[j] * g0;
    for (int ax = 0; ax < 3; ax++) acc[ax] += -P->G * mass[j] * g1 * d[ax];
}

void or_direct(const uint32_t *pos, int64_t np, const double *mass, const uint8_t *cls,
               const int64_t *sinks, int64_t ns, const or_params *P, double r_max,
               double *acc, double *pot)
{
    double r2max = r_max > 0 ? r_max * r_max : 0.0;
    int use_cells = P->periodic && r_max > 0 && r_max * 3.0 <= P->box;
    if (!use_cells) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t s = 0; s < ns; s++) {
            int64_t i = sinks[s];
            double a[3] = {0, 0, 0}, ph = 0.0;
            for (int64_t j = 0; j < np; j++)
                if (j != i) or_pair_acc(pos, np, mass, cls, i, j, P, a, &ph, r2max);
            for (int ax = 0; ax < 3; ax++) acc[3 * s + ax] = a[ax];
            pot[s] = ph;
        }
        return;
    }
    /* cell list: cells of side >= r_max, sources bucketed by cell (a filter only) */
    int nc = (int)floor(P->box / r_max);
    if (nc > 512) nc = 512;
    int64_t ncell = (int64_t)nc * nc * nc;
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (ncell + 1));
    int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (np > 0 ? np : 1));
    int64_t *cell_of = (int64_t *)malloc(sizeof(int64_t) * (np > 0 ? np : 1));
    for (int64_t c = 0; c <= ncell; c++) head[c] = 0;
    for (int64_t j = 0; j < np; j++) {
        int64_t c[3];
        for (int ax = 0; ax < 3; ax++) {
            c[ax] = (int64_t)((double)pos[ax * np + j] / 4294967296.0 * nc);
            if (c[ax] >= nc) c[ax] = nc - 1;
        }
        cell_of[j] = (c[0] * nc + c[1]) * nc + c[2];
        head[cell_of[j] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) head[c + 1] += head[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (ncell > 0 ? ncell : 1));
    for (int64_t c = 0; c < ncell; c++) fill[c] = head[c];
    for (int64_t j = 0; j < np; j++) list[fill[cell_of[j]]++] = j;
    free(fill);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < ns; s++) {
        int64_t i = sinks[s];
        double a[3] = {0, 0, 0}, ph = 0.0;
        int64_t ci[3];
        for (int ax = 0; ax < 3; ax++) {
            ci[ax] = (int64_t)((double)pos[ax * np + i] / 4294967296.0 * nc);
            if (ci[ax] >= nc) ci[ax] = nc - 1;
        }
        for (int dx = -1; dx <= 1; dx++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dz = -1; dz <= 1; dz++) {
                    int64_t cx = (ci[0] + dx + nc) % nc, cy = (ci[1] + dy + nc) % nc,
                            cz = (ci[2] + dz + nc) % nc;
                    int64_t c = (cx * nc + cy) * nc + cz;
                    for (int64_t q = head[c]; q < head[c + 1]; q++) {
                        int64_t j = list[q];
                        if (j != i) or_pair_acc(pos, np, mass, cls, i, j, P, a, &ph, r2max);
                    }
                }
        for (int ax = 0; ax < 3; ax++) acc[3 * s + ax] = a[ax];
        pot[s] = ph;
    }
    free(head); free(list); free(cell_of);
}

/* ===================================================================================== */
/* a8: Cartesian FMM (Sec. 2.4, Appendix A)                                                */
/* ===================================================================================== */

/* Field tensors T_k (k = 0..p, full 3^k components) per node: the potential near the node's
 * centre of mass is Phi(s + a) = sum_k (1/k!) T_k . a^(k). */
typedef struct {
    const or_tree *t;
    const uint32_t *pos;
    int64_t np;
    const double *mass;
    const uint8_t *cls;
    const double *aold;
    const or_params *P;
    double *T;      /* nn x ntens */
    int ntens;
    int toff[OR_MAXP + 2];
    double *acc, *pot;
    int64_t *pcnt;  /* per particle: particle-particle and particle-node interactions (or NULL) */
    int64_t n_m2l, n_pn, n_p2p;
} or_fmm_ctx;

/* A cell of the dual walk: a tree node, or a single particle.  Sec. 2.4 lets the walk pair
 * nodes with nodes or with single particles; a particle is a cell of side 0 centred on itself
 * whose only moment is Q_0 = m (its dipole and higher moments about its own position
 * vanish). */
typedef struct {
    int64_t k;   /* node index, or sorted particle index */
    int part;    /* 1: particle */
} or_cell;

static int or_is_leaf(const or_tree *t, int64_t k) { return t->next[k] == k + 1; }

static double or_cell_side(const or_fmm_ctx *C, or_cell X)
{
    return X.part ? 0.0 : ldexp(C->P->box, -C->t->level[X.k]);
}

static uint32_t or_cell_centre(const or_fmm_ctx *C, or_cell X, int ax)
{
    return X.part ? C->pos[ax * C->np + X.k] : C->t->center[3 * X.k + ax];
}

static double or_cell_com(const or_fmm_ctx *C, or_cell X, int ax)
{
    return X.part ? 0.0 : C->t->com[3 * X.k + ax];   /* s - geometric centre */
}

static double or_cell_mass(const or_fmm_ctx *C, or_cell X)
{
    return X.part ? C->mass[X.k] : C->t->mass[X.k];
}

static double or_cell_eps(const or_fmm_ctx *C, or_cell X)
{
    if (!X.part) return C->t->eps_max[X.k];
    return C->P->eps[C->cls ? C->cls[X.k] : 0];
}

static double or_cell_eps_min(const or_fmm_ctx *C, or_cell X)
{
    if (!X.part) return C->t->eps_min[X.k];
    return C->P->eps[C->cls ? C->cls[X.k] : 0];
}

static double or_cell_amin(const or_fmm_ctx *C, or_cell X)
{
    if (!X.part) return C->t->amin[X.k];
    return C->aold ? C->aold[X.k] : 0.0;
}

/* symmetric particle-particle interaction of sorted particles i != j (Eqs. eqnsoft, eqnpo4) */
static void or_pp(or_fmm_ctx *C, int64_t i, int64_t j)
{
    const or_params *P = C->P;
    double d[3];
    for (int ax = 0; ax < 3; ax++)
        d[ax] = or_sep(C->pos[ax * C->np + j], C->pos[ax * C->np + i], P);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (P->r_s > 0.0 && P->pp_cut && r2 >= P->r_cut * P->r_cut) return;
    double ei = P->eps[C->cls ? C->cls[i] : 0], ej = P->eps[C->cls ? C->cls[j] : 0];
    double h = 2.8 * (ei > ej ? ei : ej), g0, g1;
    or_pair_kernel(sqrt(r2), h, P->r_s, &g0, &g1);
    C->pot[i] += -P->G * C->mass[j] * g0;
    C->pot[j] += -P->G * C->mass[i] * g0;
    for (int ax = 0; ax < 3; ax++) {
        C->acc[3 * i + ax] += -P->G * C->mass[j] * g1 * d[ax];
        C->acc[3 * j + ax] += P->G * C->mass[i] * g1 * d[ax];
    }
    if (P->ewald && P->periodic && P->r_s <= 0.0) {
        /* the Ewald correction of the pair (psi even, its gradient odd) */
        double ai[3] = {0, 0, 0}, pi_ = 0.0;
        or_pp_ewald(d, 1.0, P->box, P->G, ai, &pi_);
        C->pot[i] += C->mass[j] * pi_;
        C->pot[j] += C->mass[i] * pi_;
        for (int ax = 0; ax < 3; ax++) {
            C->acc[3 * i + ax] += C->mass[j] * ai[ax];
            C->acc[3 * j + ax] -= C->mass[i] * ai[ax];
        }
    }
    C->n_p2p++;
    if (C->pcnt) { C->pcnt[2 * i]++; C->pcnt[2 * j]++; }
}

/* Field tensors of the mutual expansion of two cells with moments QA, QB (monomials of orders
 * 0..p about their centres of mass) and r = s_B - s_A (Sec. 2.4):
 *   fA_k = -G (-1)^k sum_{n=0}^{p-k} (1/n!) D_{n+k}(r) . Q^B_n      (field of B around s_A)
 *   fB_k = -G        sum_{n=0}^{p-k} ((-1)^n/n!) D_{n+k}(r) . Q^A_n (field of A around s_B)
 * Q_p is dropped unless keep_qp is set (it only shifts the potential by a constant).  h > 0
 * takes the derivatives of the softened kernel with h = 2.8 eps_ij (or_gn_soft) instead of
 * the unsoftened ones.  fA, fB: full tensors of orders 0..p at offsets toff[k]. */
static void or_m2l_fields(const double *QA, const double *QB, const double *rv, int p,
                          double r_s, double h, double G, int keep_qp, const int *toff,
                          double *fA, double *fB, double L_ewald)
{
    double r = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
    double g[OR_MAXP + 2];
    if (h > 0.0) or_gn_soft(r, h, r_s, p, g);   /* softened multipoles (Sec. 2.7) */
    else or_gn(r, r_s, p, g);
    static __thread double D[OR_MAXP + 1][729];
    for (int m = 0; m <= p; m++) or_D_full(m, rv, g, D[m]);
    if (L_ewald > 0.0) {
        /* pure periodic FMM (Sec. 2.2.4): the kernel is 1/r - psi, the correction expanded
         * with the same tensors */
        static __thread double Dp[OR_EW_MMAX + 1][729];
        or_ewald_dpsi(rv, L_ewald, p, Dp);
        for (int m = 0; m <= p; m++)
            for (int t = 0; t < or_pow3(m); t++) D[m][t] -= Dp[m][t];
    }
    for (int k = 0; k <= p; k++) {
        int k3 = or_pow3(k);
        double sk = (k & 1) ? -1.0 : 1.0;
        for (int I = 0; I < k3; I++) {
            double fa = 0.0, fb = 0.0;
            for (int n = 0; n <= p - k; n++) {
                if (n == p && !keep_qp) continue;
                double inv = 1.0 / or_factorial(n), sn = (n & 1) ? -1.0 : 1.0;
                int n3 = or_pow3(n);
                for (int J = 0; J < n3; J++) {
                    double d = D[n + k][I + k3 * J];
                    fa += inv * d * or_Q_full(QB, n, J);
                    fb += inv * sn * d * or_Q_full(QA, n, J);
                }
            }
            fA[toff[k] + I] = -G * sk * fa;
            fB[toff[k] + I] = -G * fb;
        }
    }
}

/* Adds a field to a cell: a node keeps it for the downward pass; a particle evaluates it at
 * its own position (a = 0): potential T_0, acceleration -T_1. */
static void or_deposit(or_fmm_ctx *C, or_cell X, const double *f)
{
    if (X.part) {
        C->pot[X.k] += f[C->toff[0]];
        for (int ax = 0; ax < 3; ax++) C->acc[3 * X.k + ax] += -f[C->toff[1] + ax];
        return;
    }
    double *T = C->T + (int64_t)C->ntens * X.k;
    for (int c = 0; c < C->ntens; c++) T[c] += f[c];
}

/* Accepted interaction of two cells, both directions (node-node or particle-node); h > 0 for a
 * softened interaction. */
static void or_m2l(or_fmm_ctx *C, or_cell A, or_cell B, const double *rv, double h)
{
    const or_tree *t = C->t;
    const or_params *P = C->P;
    int64_t nm = or_nmono(t->order);
    static __thread double QpA[OR_MAXP * 64], QpB[OR_MAXP * 64], fA[800], fB[800];
    const double *QA, *QB;
    if (A.part) {
        for (int64_t c = 0; c < nm; c++) QpA[c] = 0.0;
        QpA[0] = C->mass[A.k];
        QA = QpA;
    } else {
        QA = t->mono + nm * A.k;
    }
    if (B.part) {
        for (int64_t c = 0; c < nm; c++) QpB[c] = 0.0;
        QpB[0] = C->mass[B.k];
        QB = QpB;
    } else {
        QB = t->mono + nm * B.k;
    }
    or_m2l_fields(QA, QB, rv, P->order, P->r_s, h, P->G, P->keep_qp, C->toff, fA, fB,
                  (P->ewald && P->periodic && P->r_s <= 0.0) ? P->box : 0.0);
    or_deposit(C, A, fA);
    or_deposit(C, B, fB);
    if (A.part || B.part) {
        C->n_pn++;
        if (C->pcnt) C->pcnt[2 * (A.part ? A.k : B.k) + 1]++;
    } else {
        C->n_m2l++;
    }
}

static void or_interact(or_fmm_ctx *C, or_cell A, or_cell B);

/* all pairs of the daughters of X (a leaf's daughters are its particles), each pair once */
static void or_self(or_fmm_ctx *C, or_cell X)
{
    const or_tree *t = C->t;
    if (X.part) return;   /* a particle has no self-interaction */
    int64_t k = X.k;
    if (or_is_leaf(t, k)) {
        for (int64_t i = t->first[k]; i < t->first[k] + t->count[k]; i++)
            for (int64_t j = i + 1; j < t->first[k] + t->count[k]; j++) {
                or_cell a = {i, 1}, b = {j, 1};
                or_interact(C, a, b);
            }
        return;
    }
    for (int64_t c1 = k + 1; c1 < t->next[k]; c1 = t->next[c1])
        for (int64_t c2 = c1; c2 < t->next[k]; c2 = t->next[c2]) {
            or_cell a = {c1, 0}, b = {c2, 0};
            if (c1 == c2) or_self(C, a);
            else or_interact(C, a, b);
        }
}

/* daughters of node X: child nodes, or the particles of a leaf */
static int64_t or_daughters(const or_fmm_ctx *C, int64_t k, or_cell **out)
{
    const or_tree *t = C->t;
    int64_t n = 0;
    if (or_is_leaf(t, k)) {
        *out = (or_cell *)malloc(sizeof(or_cell) * (size_t)(t->count[k] > 0 ? t->count[k] : 1));
        for (int64_t i = t->first[k]; i < t->first[k] + t->count[k]; i++) {
            (*out)[n].k = i;
            (*out)[n].part = 1;
            n++;
        }
        return n;
    }
    *out = (or_cell *)malloc(sizeof(or_cell) * 8);
    for (int64_t c = k + 1; c < t->next[k]; c = t->next[c]) {
        (*out)[n].k = c;
        (*out)[n].part = 0;
        n++;
    }
    return n;
}

/* Dual tree walk (Sec. 2.4) over cells A != B: a pair either interacts through the symmetric
 * expansion (fields added to both cells), or is opened.  Readings:
 *   - two particles always interact directly (pair kernel, softened);
 *   - a failing pair opens both of its cells; a particle cannot be opened, so a
 *     particle paired with a node opens the node only; a leaf opens into its particles, which
 *     then meet the other side's daughters as particle-node pairs (the cell-particle
 *     interactions of the method's second phase);
 *   - pairs whose nearest faces are further apart than r_cut are dropped (Sec. 2.5); for a
 *     particle the "cube" is its position;
 *   - in a periodic box the centres are taken at their nearest images and then the centre-of-
 *     mass separation at its own nearest image (so both cells see the same image);
 *   - with the exclusion zone on, a pair does not interact when the centre separation is
 *     within max(l_A, l_B) along every axis: touching equal-sized nodes, or a particle inside
 *     the exclusion cube of side 2l around a node (the tree's zone, Sec. 2.2.3); overlapping
 *     cubes never interact;
 *   - a pair with r < 2.8 eps_ij, eps_ij = max(eps_max(A), eps_max(B)), is opened under the
 *     GADGET-3 rule (multipoles unsoftened); under the GADGET-4 rule of Sec. 2.7 only if
 *     eps_min(A) < eps_ij and eps_min(B) < eps_ij (both cells mixed), otherwise the pair
 *     interacts through the expansion of the softened kernel with eps_ij;
 *   - relative criterion G M_max / r^2 (l_max / r)^(p-1) < alpha min(|a|_A, |a|_B), or the
 *     geometric one (l_A + l_B) / r < theta_c (Eq. eqnNodeDec); a particle contributes its
 *     own mass, side 0, softening and |a_old|.                                              */
static void or_interact(or_fmm_ctx *C, or_cell A, or_cell B)
{
    const or_params *P = C->P;
    if (A.part && B.part) { or_pp(C, A.k, B.k); return; }
    double lA = or_cell_side(C, A), lB = or_cell_side(C, B);
    double dc[3];
    for (int ax = 0; ax < 3; ax++)
        dc[ax] = or_sep(or_cell_centre(C, B, ax), or_cell_centre(C, A, ax), P);
    if (P->r_s > 0.0) {
        double e2 = 0.0;
        for (int ax = 0; ax < 3; ax++) {
            double e = fabs(dc[ax]) - 0.5 * (lA + lB);
            if (e > 0) e2 += e * e;
        }
        if (e2 > P->r_cut * P->r_cut) return;
    }
    double rv[3];
    for (int ax = 0; ax < 3; ax++) rv[ax] = dc[ax] + or_cell_com(C, B, ax) - or_cell_com(C, A, ax);
    if (P->periodic)   /* the nearest image of the centre-of-mass separation */
        for (int ax = 0; ax < 3; ax++) rv[ax] -= P->box * rint(rv[ax] / P->box);
    double r2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
    int accept = 1;
    double dmax = fmax(fabs(dc[0]), fmax(fabs(dc[1]), fabs(dc[2])));
    if (P->exclusion && dmax <= fmax(lA, lB)) accept = 0;   /* touching / exclusion zone */
    if (dmax < 0.5 * (lA + lB)) accept = 0;                  /* overlapping cubes */
    double em = fmax(or_cell_eps(C, A), or_cell_eps(C, B)), hsoft = 0.0;
    if (r2 < (2.8 * em) * (2.8 * em)) {
        if (!P->soft_nodes) accept = 0;
        else if (or_cell_eps_min(C, A) < em && or_cell_eps_min(C, B) < em) accept = 0;
        else hsoft = 2.8 * em;
    }
    if (accept) {
        if (P->criterion == 1) {
            if ((lA + lB) * (lA + lB) >= P->theta * P->theta * r2) accept = 0;
        } else {
            double r = sqrt(r2);
            double Mmax = fmax(or_cell_mass(C, A), or_cell_mass(C, B)), lmax = fmax(lA, lB);
            double amin = fmin(or_cell_amin(C, A), or_cell_amin(C, B));
            double lhs = P->G * Mmax * or_ipow(lmax, P->order - 1);
            double rhs = P->alpha * amin * or_ipow(r, P->order + 1);
            if (!(lhs < rhs)) accept = 0;
        }
    }
    if (accept) { or_m2l(C, A, B, rv, hsoft); return; }
    or_cell *da = NULL, *db = NULL;
    int64_t na = 1, nb = 1;
    if (!A.part) na = or_daughters(C, A.k, &da);
    if (!B.part) nb = or_daughters(C, B.k, &db);
    for (int64_t u = 0; u < na; u++)
        for (int64_t v = 0; v < nb; v++)
            or_interact(C, da ? da[u] : A, db ? db[v] : B);
    free(da);
    free(db);
}

/* contraction of a full order-(k+j) tensor with v^(j) over its last j slots */
static double or_contract_tail(const double *Tkj, int k, int j, int I, const double *v)
{
    int k3 = or_pow3(k), j3 = or_pow3(j);
    double s = 0.0;
    for (int J = 0; J < j3; J++) {
        double vp = 1.0;
        int w = J;
        for (int u = 0; u < j; u++) { vp *= v[w % 3]; w /= 3; }
        s += Tkj[I + k3 * J] * vp;
    }
    return s;
}

/* Evaluation of a field T (full tensors of orders 0..p at toff) at offset a from its centre:
 * Phi = sum_k (1/k!) T_k . a^(k),  grad Phi = sum_{k>=1} (1/(k-1)!) T_k . a^(k-1). */
static void or_l2p(const double *T, const int *toff, int p, const double *a, double *phi,
                   double *grad)
{
    double ph = 0.0;
    for (int q = 0; q <= p; q++) {
        int q3 = or_pow3(q);
        double inv = 1.0 / or_factorial(q);
        for (int I = 0; I < q3; I++) {
            double ap = 1.0;
            int w = I;
            for (int u = 0; u < q; u++) { ap *= a[w % 3]; w /= 3; }
            ph += inv * T[toff[q] + I] * ap;
        }
    }
    *phi = ph;
    for (int ax = 0; ax < 3; ax++) {
        double s = 0.0;
        for (int q = 1; q <= p; q++)
            s += or_contract_tail(T + toff[q], 1, q - 1, ax, a) / or_factorial(q - 1);
        grad[ax] = s;
    }
}

/* Downward pass (Sec. 2.4, phase 3): the parent field is shifted to each daughter's centre
 * of mass, T^C_k += sum_j (1/j!) T^P_{k+j} . d^(j) with d = s_C - s_P, and at the leaves
 * evaluated at the particles (or_l2p with a = x - s; acceleration = -grad Phi).           */
static void or_down(or_fmm_ctx *C, int64_t k)
{
    const or_tree *t = C->t;
    const or_params *P = C->P;
    int p = P->order;
    double scale = P->box / 4294967296.0;
    double *Tp = C->T + (int64_t)C->ntens * k;
    if (or_is_leaf(t, k)) {
        for (int64_t i = t->first[k]; i < t->first[k] + t->count[k]; i++) {
            double a[3], phi, grad[3];
            for (int ax = 0; ax < 3; ax++)
                a[ax] = or_isep(C->pos[ax * C->np + i], t->center[3 * k + ax], 0) * scale
                        - t->com[3 * k + ax];
            or_l2p(Tp, C->toff, p, a, &phi, grad);
            C->pot[i] += phi;
            for (int ax = 0; ax < 3; ax++) C->acc[3 * i + ax] += -grad[ax];
        }
        return;
    }
    for (int64_t c = k + 1; c < t->next[k]; c = t->next[c]) {
        double d[3];
        for (int ax = 0; ax < 3; ax++)
            d[ax] = or_isep(t->center[3 * c + ax], t->center[3 * k + ax], 0) * scale
                    + t->com[3 * c + ax] - t->com[3 * k + ax];
        double *Tc = C->T + (int64_t)C->ntens * c;
        for (int q = 0; q <= p; q++) {
            int q3 = or_pow3(q);
            for (int I = 0; I < q3; I++) {
                double s = 0.0;
                for (int j = 0; j <= p - q; j++)
                    s += or_contract_tail(Tp + C->toff[q + j], q, j, I, d) / or_factorial(j);
                Tc[C->toff[q] + I] += s;
            }
        }
        or_down(C, c);
    }
}

static int or_tensor_offsets(int p, int *toff)
{
    int off = 0;
    for (int k = 0; k <= p; k++) { toff[k] = off; off += or_pow3(k); }
    return off;
}

/* Full FMM force computation for all particles (sorted order).  acc: n x 3, pot: n.
 * aold: |a_old| per sorted particle (relative criterion; NULL = 0).
 * counts[0] = node-node expansions, counts[1] = particle-node expansions, counts[2] = particle
 * pairs (each unordered pair once).  pcounts (n x 2, nullable): per particle, the particle
 * pairs and the particle-node expansions it takes part in. */
void or_fmm(const or_tree *t, const uint32_t *pos, int64_t np, const double *mass,
            const uint8_t *cls, const double *aold, const or_params *P, double *acc,
            double *pot, int64_t *counts, int64_t *pcounts)
{
    or_fmm_ctx C;
    memset(&C, 0, sizeof(C));
    C.t = t; C.pos = pos; C.np = np; C.mass = mass; C.cls = cls; C.aold = aold; C.P = P;
    C.acc = acc; C.pot = pot; C.pcnt = pcounts;
    C.ntens = or_tensor_offsets(P->order, C.toff);
    C.T = (double *)calloc((size_t)C.ntens * (size_t)(t->nn ? t->nn : 1), sizeof(double));
    for (int64_t i = 0; i < 3 * np; i++) acc[i] = 0.0;
    for (int64_t i = 0; i < np; i++) pot[i] = 0.0;
    if (pcounts)
        for (int64_t i = 0; i < 2 * np; i++) pcounts[i] = 0;
    if (t->nn > 0) {
        or_cell root = {0, 0};
        or_self(&C, root);   /* the root interacting with itself */
        or_down(&C, 0);
    }
    if (P->ewald && P->periodic && P->r_s <= 0.0) {   /* each particle's own images */
        const double z[3] = {0.0, 0.0, 0.0};
        const double psi0 = or_ewald_psi(z, P->box, 2.0 / P->box, 2, 5);
        for (int64_t i = 0; i < np; i++) pot[i] += P->G * mass[i] * psi0;
    }
    counts[0] = C.n_m2l;
    counts[1] = C.n_pn;
    counts[2] = C.n_p2p;
    free(C.T);
}

/* ===================================================================================== */
/* Two-node expansion test harness (Sec. 3.1): the particles of two groups A and B, given in */
/* physical coordinates (n x 3), interact only through one expansion.                     */
/* ===================================================================================== */

/* Monomial moments of orders 0..p about the centre of mass, by definition (Sec. 2.2.2). */
void or_moments_points(const double *x, const double *m, int64_t n, int p, double *com,
                       double *mono)
{
    double M = 0.0, d[3] = {0, 0, 0};
    for (int64_t j = 0; j < n; j++) {
        M += m[j];
        for (int ax = 0; ax < 3; ax++) d[ax] += m[j] * x[3 * j + ax];
    }
    for (int ax = 0; ax < 3; ax++) com[ax] = d[ax] / M;
    int64_t nm = or_nmono(p);
    for (int64_t c = 0; c < nm; c++) mono[c] = 0.0;
    for (int64_t j = 0; j < n; j++) {
        double dx[3];
        for (int ax = 0; ax < 3; ax++) dx[ax] = x[3 * j + ax] - com[ax];
        for (int q = 0; q <= p; q++)
            for (int a = q; a >= 0; a--)
                for (int b = q - a; b >= 0; b--) {
                    int c = q - a - b;
                    mono[or_mono_index(a, b, c)] +=
                        m[j] * or_ipow(dx[0], a) * or_ipow(dx[1], b) * or_ipow(dx[2], c);
                }
    }
}

/* The particle-node term of the softened kernel (or_pn_h with h = 2.8 eps), exported for pins. */
void or_pn_soft_eval(const double *mono, const double *rv, int p, double r_s, double h, double G,
                     double *acc, double *pot)
{
    acc[0] = acc[1] = acc[2] = 0.0;
    *pot = 0.0;
    or_pn_h(mono, rv, p, r_s, h, G, acc, pot);
}

/* One-sided tree: the particle-node term (or_pn) of group B at every particle of A. */
void or_two_node_tree(const double *xa, int64_t na, const double *xb, const double *mb,
                      int64_t nb, int p, double r_s, double G, double *acc, double *pot)
{
    double com[3], mono[64];
    or_moments_points(xb, mb, nb, p, com, mono);
    for (int64_t i = 0; i < na; i++) {
        double rv[3];
        for (int ax = 0; ax < 3; ax++) rv[ax] = com[ax] - xa[3 * i + ax];
        acc[3 * i] = acc[3 * i + 1] = acc[3 * i + 2] = 0.0;
        pot[i] = 0.0;
        or_pn(mono, rv, p, r_s, G, acc + 3 * i, pot + i);
    }
}

/* FMM: the mutual expansion of A and B (or_m2l_fields), each field evaluated at its own
 * group's particles (or_l2p); outputs for A's particles then B's. */
void or_two_node_fmm(const double *xa, const double *ma, int64_t na, const double *xb,
                     const double *mb, int64_t nb, int p, double r_s, double G, int keep_qp,
                     double *acc_a, double *pot_a, double *acc_b, double *pot_b)
{
    double sA[3], sB[3], QA[64], QB[64], rv[3];
    int toff[OR_MAXP + 2];
    int nt = or_tensor_offsets(p, toff);
    double *fA = (double *)calloc((size_t)nt, sizeof(double));
    double *fB = (double *)calloc((size_t)nt, sizeof(double));
    or_moments_points(xa, ma, na, p, sA, QA);
    or_moments_points(xb, mb, nb, p, sB, QB);
    for (int ax = 0; ax < 3; ax++) rv[ax] = sB[ax] - sA[ax];
    or_m2l_fields(QA, QB, rv, p, r_s, 0.0, G, keep_qp, toff, fA, fB, 0.0);
    for (int64_t i = 0; i < na; i++) {
        double a[3], grad[3];
        for (int ax = 0; ax < 3; ax++) a[ax] = xa[3 * i + ax] - sA[ax];
        or_l2p(fA, toff, p, a, pot_a + i, grad);
        for (int ax = 0; ax < 3; ax++) acc_a[3 * i + ax] = -grad[ax];
    }
    for (int64_t i = 0; i < nb; i++) {
        double a[3], grad[3];
        for (int ax = 0; ax < 3; ax++) a[ax] = xb[3 * i + ax] - sB[ax];
        or_l2p(fB, toff, p, a, pot_b + i, grad);
        for (int ax = 0; ax < 3; ax++) acc_b[3 * i + ax] = -grad[ax];
    }
    free(fA);
    free(fB);
}

/* ===================================================================================== */
/* Periodic point-mass potential and force by Ewald summation (Sec. 2.1, Eq. eqnewal): the   */
/* exact reference for the long-range (PM) part of the TreePM split, Sec. 2.3.             */
/* ===================================================================================== */

/* Sum over real-space images n with |n_i| <= nr and over wave vectors k = 2 pi m / L,
 * m != 0, |m_i| <= nk.  alpha: the Ewald split parameter (any value; the result does not
 * depend on it once both sums have converged). */

/* Correction potential psi(x) of Eq. (eqnewal) for a cubic box of side L:
 *   psi = 1/|x| + pi/(alpha^2 V) - sum_n erfc(alpha |x + q_n|)/|x + q_n|
 *         - (4 pi / V) sum_{k != 0} exp(-k^2 / (4 alpha^2)) / k^2 cos(k . x),
 * with the n = 0 term combined with 1/|x| as erf(alpha |x|)/|x| (finite at x = 0). */
double or_ewald_psi(const double *x, double L, double alpha, int nr, int nk)
{
    const double V = L * L * L, pi = 3.14159265358979323846;
    double r0 = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    double s = (r0 > 0.0) ? erf(alpha * r0) / r0 : 2.0 * alpha / sqrt(pi);
    s += pi / (alpha * alpha * V);
    for (int a = -nr; a <= nr; a++)
        for (int b = -nr; b <= nr; b++)
            for (int c = -nr; c <= nr; c++) {
                if (a == 0 && b == 0 && c == 0) continue;
                double d[3] = {x[0] + a * L, x[1] + b * L, x[2] + c * L};
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                s -= erfc(alpha * r) / r;
            }
    for (int a = -nk; a <= nk; a++)
        for (int b = -nk; b <= nk; b++)
            for (int c = -nk; c <= nk; c++) {
                if (a == 0 && b == 0 && c == 0) continue;
                double k[3] = {2 * pi * a / L, 2 * pi * b / L, 2 * pi * c / L};
                double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                s -= 4 * pi / V * exp(-k2 / (4 * alpha * alpha)) / k2 *
                     cos(k[0] * x[0] + k[1] * x[1] + k[2] * x[2]);
            }
    return s;
}

/* Acceleration of a unit test mass at x due to a unit point mass at the origin in the
 * periodic box (with the neutralising background), a = -grad Phi with
 * Phi(x) = pi/(alpha^2 V) - sum_n erfc(alpha s_n)/s_n - (4 pi/V) sum_k e^{-k^2/4alpha^2}/k^2 cos(k.x),
 * s_n = |x + q_n|:
 *   a = - sum_n s_vec [erfc(alpha s) + (2 alpha s / sqrt(pi)) exp(-alpha^2 s^2)] / s^3
 *       - (4 pi / V) sum_k (k / k^2) exp(-k^2 / 4 alpha^2) sin(k . x).
 * kspace_only = 1 returns only the second sum: with alpha = 1/(2 r_s) that is the exact
 * long-range force of the TreePM split (the Fourier sum of Eq. eqnksum). */
void or_ewald_force(const double *x, double L, double alpha, int nr, int nk, int kspace_only,
                    double *acc)
{
    const double V = L * L * L, pi = 3.14159265358979323846;
    acc[0] = acc[1] = acc[2] = 0.0;
    if (!kspace_only)
        for (int a = -nr; a <= nr; a++)
            for (int b = -nr; b <= nr; b++)
                for (int c = -nr; c <= nr; c++) {
                    double d[3] = {x[0] + a * L, x[1] + b * L, x[2] + c * L};
                    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    if (r == 0.0) continue;
                    double f = (erfc(alpha * r) + 2.0 * alpha * r / sqrt(pi) * exp(-alpha * alpha * r * r))
                               / (r * r * r);
                    for (int i = 0; i < 3; i++) acc[i] -= f * d[i];
                }
    for (int a = -nk; a <= nk; a++)
        for (int b = -nk; b <= nk; b++)
            for (int c = -nk; c <= nk; c++) {
                if (a == 0 && b == 0 && c == 0) continue;
                double k[3] = {2 * pi * a / L, 2 * pi * b / L, 2 * pi * c / L};
                double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                double f = 4 * pi / V * exp(-k2 / (4 * alpha * alpha)) / k2 *
                           sin(k[0] * x[0] + k[1] * x[1] + k[2] * x[2]);
                for (int i = 0; i < 3; i++) acc[i] -= f * k[i];
            }
}

/* g_n = (r^-1 d/dr)^n of erf(alpha r) / r, n = 0..nmax.  With erf(a r)/r =
 * (2 a/sqrt(pi)) sum_k (-1)^k (a r)^(2k) / (k! (2k+1)) and (r^-1 d/dr) r^(2k) = 2k r^(2k-2):
 *   g_n = (-1)^n (2/sqrt(pi)) 2^n a^(2n+1) sum_j (-1)^j (a r)^(2j) / (j! (2j+2n+1)),
 * summed for a r < 1.5; beyond, g_n of 1/r minus g_n of erfc(a r)/r (or_gn with
 * r_s = 1/(2a)), where the two no longer cancel badly. */
static void or_gn_erf(double r, double alpha, int nmax, double *g)
{
    const double pi = 3.14159265358979323846;
    const double x = alpha * r;
    if (x < 1.5) {
        double pre = 2.0 / sqrt(pi) * alpha;
        for (int n = 0; n <= nmax; n++) {
            double s = 0.0, term = 1.0;   /* (-1)^j x^(2j) / j! */
            for (int j = 0; j < 60; j++) {
                s += term / (2.0 * j + 2.0 * n + 1.0);
                term *= -x * x / (j + 1.0);
            }
            g[n] = ((n & 1) ? -1.0 : 1.0) * pre * s;
            pre *= 2.0 * alpha * alpha;
        }
        return;
    }
    double gN[OR_EW_MMAX + 2], gE[OR_EW_MMAX + 2];
    or_gn(r, 0.0, nmax, gN);
    or_gn(r, 0.5 / alpha, nmax, gE);
    for (int n = 0; n <= nmax; n++) g[n] = gN[n] - gE[n];
}

/* Full derivative tensors D_m[psi](x), m = 0..mmax (<= OR_EW_MMAX), of the correction
 * potential psi of Eq. (eqnewal) for a cubic box of side L (Sec. 2.2.4), for separations in
 * the primary cell (|x_i| <= L/2, as nearest-image separations are), term by term:
 *   psi = pi/(a^2 V) + erf(a|x|)/|x| - sum_{n != 0} erfc(a|x+q_n|)/|x+q_n|
 *         - (4 pi/V) sum_{k != 0} exp(-k^2/(4 a^2))/k^2 cos(k . x),
 * radial terms through g_n and the pairing formula (or_D_full), the Fourier terms through
 * d/dx_i cos(k.x + phase) = k_i cos(k.x + phase + pi/2), k and -k together (their terms are
 * equal).  a = 3.5/L with |n_i| <= 1 (the first image left out lies beyond 1.5 L: erfc(5.25)
 * ~ 1e-13) and |m_i| <= 7 (k = 2 pi m/L; exp(-pi^2 m^2/(aL)^2) ~ 1e-17 at m = 7). */
#define OR_EW_NK 7
void or_ewald_dpsi(const double *x, double L, int mmax, double (*D)[729])
{
    const double pi = 3.14159265358979323846, V = L * L * L, alpha = 3.5 / L;
    const int nr = 1, nk = OR_EW_NK;
    /* the half space of wave vectors with their weights, cached per thread for the last L */
    enum { NKH = ((2 * OR_EW_NK + 1) * (2 * OR_EW_NK + 1) * (2 * OR_EW_NK + 1) - 1) / 2 };
    static __thread double kc_L = -1.0, kc_k[NKH][3], kc_w[NKH];
    if (kc_L != L) {
        int q = 0;
        for (int a = -nk; a <= nk; a++)
            for (int b = -nk; b <= nk; b++)
                for (int c = -nk; c <= nk; c++) {
                    /* one of each pair k, -k: the first non-zero index positive */
                    if (!(a > 0 || (a == 0 && (b > 0 || (b == 0 && c > 0))))) continue;
                    double k[3] = {2 * pi * a / L, 2 * pi * b / L, 2 * pi * c / L};
                    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                    for (int i = 0; i < 3; i++) kc_k[q][i] = k[i];
                    kc_w[q] = 2.0 * 4 * pi / V * exp(-k2 / (4 * alpha * alpha)) / k2;
                    q++;
                }
        kc_L = L;
    }
    double g[OR_EW_MMAX + 2], tmp[729];
    for (int m = 0; m <= mmax; m++)
        for (int t = 0; t < or_pow3(m); t++) D[m][t] = 0.0;
    D[0][0] = pi / (alpha * alpha * V);
    for (int a = -nr; a <= nr; a++)
        for (int b = -nr; b <= nr; b++)
            for (int c = -nr; c <= nr; c++) {
                double d[3] = {x[0] + a * L, x[1] + b * L, x[2] + c * L};
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                double sgn = 1.0;
                if (a == 0 && b == 0 && c == 0) {
                    or_gn_erf(r, alpha, mmax, g);
                } else {
                    or_gn(r, 0.5 / alpha, mmax, g);
                    sgn = -1.0;
                }
                for (int m = 0; m <= mmax; m++) {
                    or_D_full(m, d, g, tmp);
                    for (int t = 0; t < or_pow3(m); t++) D[m][t] += sgn * tmp[t];
                }
            }
    for (int q = 0; q < NKH; q++) {
        const double *k = kc_k[q];
        double th = k[0] * x[0] + k[1] * x[1] + k[2] * x[2];
        double cs[4] = {cos(th), 0.0, 0.0, 0.0};
        cs[1] = -sin(th);        /* cos(th + pi/2) */
        cs[2] = -cs[0];          /* cos(th + pi) */
        cs[3] = -cs[1];          /* cos(th + 3 pi/2) */
        for (int m = 0; m <= mmax; m++) {
            double cm = kc_w[q] * cs[m & 3];
            for (int t = 0; t < or_pow3(m); t++) {
                double prod = 1.0;
                int v = t;
                for (int u = 0; u < m; u++) { prod *= k[v % 3]; v /= 3; }
                D[m][t] -= prod * cm;
            }
        }
    }
}

/* Exact periodic forces and potentials with softened nearest-image pairs (Eq. eqnpo1): for
 * each sink i, sum_{j != i} m_j [pair kernel of the nearest image, psi correction] plus
 * m_i psi(0) in the potential: the reference of the Ewald-corrected pure periodic tree. */
void or_ewald_direct(const uint32_t *pos, int64_t np, const double *mass, const uint8_t *cls,
                     const int64_t *sinks, int64_t ns, const or_params *P, double *acc,
                     double *pot)
{
    const double z[3] = {0.0, 0.0, 0.0};
    const double psi0 = or_ewald_psi(z, P->box, 2.0 / P->box, 2, 5);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t s = 0; s < ns; s++) {
        int64_t i = sinks[s];
        double a[3] = {0, 0, 0}, ph = P->G * mass[i] * psi0;
        for (int64_t j = 0; j < np; j++) {
            if (j == i) continue;
            or_pair_acc(pos, np, mass, cls, i, j, P, a, &ph, 0.0);
            double d[3];
            for (int ax = 0; ax < 3; ax++) d[ax] = or_sep(pos[ax * np + j], pos[ax * np + i], P);
            or_pp_ewald(d, mass[j], P->box, P->G, a, &ph);
        }
        for (int ax = 0; ax < 3; ax++) acc[3 * s + ax] = a[ax];
        pot[s] = ph;
    }
}

/* D_m[psi](x) for m = 0..mmax as full tensors concatenated (1 + 3 + 9 + ... entries). */
void or_ewald_dpsi_flat(const double *x, double L, int mmax, double *out)
{
    static __thread double D[OR_EW_MMAX + 1][729];
    or_ewald_dpsi(x, L, mmax, D);
    int64_t o = 0;
    for (int m = 0; m <= mmax; m++)
        for (int t = 0; t < or_pow3(m); t++) out[o++] = D[m][t];
}

/* Many evaluations: acc[i] = sum_j m_j a(x_i - y_j) (OpenMP over the evaluation points). */
void or_ewald_force_many(const double *xe, int64_t ne, const double *ys, const double *m,
                         int64_t ns, double L, double alpha, int nr, int nk, int kspace_only,
                         double *acc)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < ne; i++) {
        double s[3] = {0, 0, 0};
        for (int64_t j = 0; j < ns; j++) {
            double d[3], a[3];
            for (int ax = 0; ax < 3; ax++) d[ax] = xe[3 * i + ax] - ys[3 * j + ax];
            or_ewald_force(d, L, alpha, nr, nk, kspace_only, a);
            for (int ax = 0; ax < 3; ax++) s[ax] += m[j] * a[ax];
        }
        for (int ax = 0; ax < 3; ax++) acc[3 * i + ax] = s[ax];
    }
}
