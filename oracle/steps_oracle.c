/*
 * steps_oracle.c -- plain, serial CPU reference of the Parallel STEPS
 * operator-splitting method (Chen & De Schutter, "Parallel STEPS", §2).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library. It shares no code
 * with the CUDA path (no headers, helpers or tables): both are written from
 * the same definitions, and the places where the two must agree bit for bit
 * (random-number layout, fixed-point thresholds, uniform construction, the
 * float logarithm of the kernel-precision mode) are spelled out here again.
 *
 * What it computes, per diffusion window (Algorithm 1, one MPI process that
 * hosts every tet, so all diffusion is "local diffusion"):
 *   1. reaction SSA operator: in every tet independently, Gillespie's direct
 *      method for the window tau, tracking the time-weighted occupancy O_S of
 *      every species changed by a fired reaction (§2.2, Algorithm 1);
 *   2. diffusion operator: for every diffusive species S in every tet, the
 *      mean occupancy Nbar = O_S / tau gives the number of trial molecules,
 *      n = binomial(trials, tau * d_{S,tet}) of them leave, and they are
 *      distributed over the tet's face neighbours in proportion to the face
 *      rates D*A/(V*d) (Algorithm 1, diffusion operator);
 *   3. all changes are applied together (Jacobi), t += tau.
 * tau = 1 / max_{S,tet} d_{S,tet} (§2.1); the last window of a run is cut to
 * t_end - t (Algorithm 1).
 *
 * Readings of points the paper leaves open:
 *   - d_{S,tet} = sum over internal faces f of D_S * A_f / (V_tet * d_f), with
 *     d_f the distance between the two tets' barycentres; boundary faces are
 *     reflective. tau is the min over diffusive species only.
 *   - binomial(Nbar, tau, d) is Bin(M, p) with p = tau * d_{S,tet} (p <= 1 by
 *     the choice of tau; the EULER law, the default) or, as an option, with
 *     p = 1 - exp(-tau d_{S,tet}) (the EXP law: the probability that an
 *     exponential leaving time with rate d falls inside the window), and M an
 *     integer trial count: M = N_S for a species no
 *     reaction changed in the window; otherwise the occupancy integral is
 *     closed at tau and Nbar is rounded stochastically (floor + Bernoulli of
 *     the fraction) and clamped to the end-of-window count (mode OCC). Mode END
 *     uses M = N_S always.
 *   - the leaving molecules are split multinomially over internal faces in
 *     proportion to the face rates. Realised molecule by molecule: each trial
 *     molecule draws one 31-bit uniform integer x and goes through face f when
 *     x falls in [T_{f-1}, T_f), T being cumulative fixed-point thresholds
 *     (2^31 * p * cumulative face-rate share); it stays when x >= T_3. This is
 *     exactly Bin(M, p) leaving followed by Multinomial(n, g_f/G), with p and
 *     the shares quantised to 2^-31. Where x comes from: a species with fewer
 *     than ORC_BULK_MIN trial molecules in a tet takes one word per molecule
 *     from the tet's word stream (species in order); one with more takes its
 *     molecules in groups of 32, whose x are assembled from 31 bit planes
 *     (plane k is bit 30 - k of every x; bit j of the plane's word belongs to
 *     molecule j of the group). Either way x is uniform on [0, 2^31), so the
 *     law is the same.
 *   - reaction propensities: order 0 a = k N_A V, order 1 a = k N_X, order 2
 *     a = k/(N_A V) N_X N_Y, homodimer a = k/(N_A V) N_X (N_X - 1).
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXS 32
#define ORC_MAXR 32
#define ORC_AVOGADRO 6.02214076e23

enum { ORC_PURPOSE_REAC = 1, ORC_PURPOSE_ROUND = 2, ORC_PURPOSE_DIFF = 3, ORC_PURPOSE_BULK = 4 };
#define ORC_BULK_MIN 16 /* trial molecules of a species in a tet from which it draws by bit planes */
enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_MESH = -2, ORC_ERR_MODEL = -3, ORC_ERR_OOM = -4 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11), written from its published definition.         */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t key_in[2], const uint32_t ctr_in[4], uint32_t out[4])
{
    uint32_t k0 = key_in[0], k1 = key_in[1];
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u; /* Weyl key schedule */
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ x1 ^ k0;
        uint32_t n2 = hi0 ^ x3 ^ k1;
        x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Counter layout of every draw of the method: key = seed, counter =
 * (window index low 32 bits, original tet id, index within the stream,
 *  purpose << 28 | window index bits 32..59). */
static void draw4(uint64_t seed, uint64_t window, uint32_t tet, uint32_t idx, uint32_t purpose,
                  uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)window, tet, idx,
                       (purpose << 28) | ((uint32_t)(window >> 32) & 0x0FFFFFFFu)};
    orc_philox4x32_10(key, ctr, out);
}

/* Bit planes of the trial molecules of species sp in group g (molecules
 * 32g .. 32g + 31) of a tet: block blk holds planes 4 blk .. 4 blk + 3.
 * Counter = (window low 32 bits, original tet id, g << 3 | blk,
 * purpose << 28 | sp << 23 | window index bits 32..54). */
static void draw4_bulk(uint64_t seed, uint64_t window, uint32_t tet, int sp, uint32_t g, uint32_t blk,
                       uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)window, tet, (g << 3) | blk,
                       ((uint32_t)ORC_PURPOSE_BULK << 28) | ((uint32_t)sp << 23) |
                           ((uint32_t)(window >> 32) & 0x007FFFFFu)};
    orc_philox4x32_10(key, ctr, out);
}

/* Uniform in (0, 1] from the top 24 bits of a word: exact in float and double. */
static double unit24(uint32_t w) { return (double)((w >> 8) + 1u) * (1.0 / 16777216.0); }

/* Uniform in (0, 1] with 53 bits from two words: exact in double. */
static double unit53(uint32_t hi, uint32_t lo)
{
    uint64_t x = (((uint64_t)hi << 32) | lo) >> 11;
    return (double)(x + 1u) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* Natural logarithm in float arithmetic for the kernel-precision mode.     */
/* Classical atanh series: x = 2^e f with f in (sqrt(1/2), sqrt(2)],        */
/* ln f = 2 atanh(s), s = (f-1)/(f+1), summed to s^11, plus e*ln2 split in  */
/* a high part exact for small e and a low part. Every step is one IEEE     */
/* single operation, evaluated in this order with no contraction.           */
/* ------------------------------------------------------------------------ */
float orc_logf32(float x)
{
    union { float f; uint32_t u; } v;
    v.f = x;
    int e = (int)((v.u >> 23) & 0xffu) - 127;
    v.u = (v.u & 0x007fffffu) | 0x3f800000u; /* f in [1, 2) */
    float f = v.f;
    if (f > 1.41421356f) { f = f * 0.5f; e = e + 1; }
    float s = (f - 1.0f) / (f + 1.0f);
    float z = s * s;
    float p = 0.0909090909f;          /* 1/11 */
    p = p * z + 0.111111111f;         /* 1/9  */
    p = p * z + 0.142857143f;         /* 1/7  */
    p = p * z + 0.2f;                 /* 1/5  */
    p = p * z + 0.333333333f;         /* 1/3  */
    p = p * z + 1.0f;
    float lnf = (s + s) * p;
    float fe = (float)e;
    float lo = fe * 1.42860682e-06f + lnf;  /* ln2 - ln2_hi */
    return fe * 0.693145752f + lo;          /* ln2_hi = 0.693145751953125 (exact) */
}

/* ------------------------------------------------------------------------ */
/* Geometry (§2.1 "local diffusion rate"; rate formula D*A/(V*d)).          */
/* Local face f of a tet is the face opposite its local vertex f.           */
/* ------------------------------------------------------------------------ */
static const int FACE_VERTS[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

static double tet_volume(const double *a, const double *b, const double *c, const double *d)
{
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double w[3] = {d[0] - a[0], d[1] - a[1], d[2] - a[2]};
    double cx = v[1] * w[2] - v[2] * w[1];
    double cy = v[2] * w[0] - v[0] * w[2];
    double cz = v[0] * w[1] - v[1] * w[0];
    double det = u[0] * cx + u[1] * cy + u[2] * cz;
    return fabs(det) / 6.0;
}

static double tri_area(const double *p, const double *q, const double *r)
{
    double u[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
    double w[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
    double cx = u[1] * w[2] - u[2] * w[1];
    double cy = u[2] * w[0] - u[0] * w[2];
    double cz = u[0] * w[1] - u[1] * w[0];
    return 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
}

static void barycentre(const double *a, const double *b, const double *c, const double *d, double *out)
{
    for (int k = 0; k < 3; ++k) out[k] = (((a[k] + b[k]) + c[k]) + d[k]) * 0.25;
}

typedef struct { int32_t v[3]; int32_t tet; int32_t face; } face_rec;

static int cmp_face(const void *x, const void *y)
{
    const face_rec *a = (const face_rec *)x, *b = (const face_rec *)y;
    for (int k = 0; k < 3; ++k) {
        if (a->v[k] != b->v[k]) return a->v[k] < b->v[k] ? -1 : 1;
    }
    if (a->tet != b->tet) return a->tet < b->tet ? -1 : 1;
    return a->face - b->face;
}

static void sort3(int32_t *v)
{
    int32_t t;
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
    if (v[1] > v[2]) { t = v[1]; v[1] = v[2]; v[2] = t; }
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
}

/* Face neighbours by matching vertex triples: nbr[4*i + f] = tet sharing
 * local face f of tet i, or -1 on the mesh boundary. */
int orc_adjacency(int64_t nv, int64_t nt, const int32_t *tets, int32_t *nbr)
{
    face_rec *fr = (face_rec *)malloc(sizeof(face_rec) * (size_t)(4 * nt + 1));
    if (!fr) return ORC_ERR_OOM;
    for (int64_t i = 0; i < nt; ++i) {
        for (int f = 0; f < 4; ++f) {
            face_rec *r = &fr[4 * i + f];
            for (int k = 0; k < 3; ++k) {
                int32_t vi = tets[4 * i + FACE_VERTS[f][k]];
                if (vi < 0 || vi >= nv) { free(fr); return ORC_ERR_MESH; }
                r->v[k] = vi;
            }
            sort3(r->v);
            r->tet = (int32_t)i;
            r->face = f;
            nbr[4 * i + f] = -1;
        }
    }
    qsort(fr, (size_t)(4 * nt), sizeof(face_rec), cmp_face);
    int64_t j = 0;
    while (j < 4 * nt) {
        int64_t e = j + 1;
        while (e < 4 * nt && memcmp(fr[e].v, fr[j].v, sizeof(fr[j].v)) == 0) ++e;
        if (e - j > 2) { free(fr); return ORC_ERR_MESH; } /* a face of 3+ tets */
        if (e - j == 2) {
            if (fr[j].tet == fr[j + 1].tet) { free(fr); return ORC_ERR_MESH; }
            nbr[4 * fr[j].tet + fr[j].face] = fr[j + 1].tet;
            nbr[4 * fr[j + 1].tet + fr[j + 1].face] = fr[j].tet;
        }
        j = e;
    }
    free(fr);
    return ORC_OK;
}

/* Per tet: volume V (m^3); per face: area A (m^2), barycentre distance d (m)
 * and geometric rate g = A / (V d) (1/m^2) for internal faces, 0 on the
 * boundary. D_S * g is the face diffusion rate (1/s). */
int orc_geometry(int64_t nv, const double *verts, int64_t nt, const int32_t *tets,
                 int32_t *nbr, double *vol, double *area, double *dist, double *g)
{
    int rc = orc_adjacency(nv, nt, tets, nbr);
    if (rc) return rc;
    for (int64_t i = 0; i < nt; ++i) {
        const double *p[4];
        for (int k = 0; k < 4; ++k) p[k] = verts + 3 * (int64_t)tets[4 * i + k];
        vol[i] = tet_volume(p[0], p[1], p[2], p[3]);
        if (!(vol[i] > 0.0)) return ORC_ERR_MESH;
    }
    for (int64_t i = 0; i < nt; ++i) {
        const double *p[4];
        for (int k = 0; k < 4; ++k) p[k] = verts + 3 * (int64_t)tets[4 * i + k];
        double ci[3];
        barycentre(p[0], p[1], p[2], p[3], ci);
        for (int f = 0; f < 4; ++f) {
            area[4 * i + f] = tri_area(p[FACE_VERTS[f][0]], p[FACE_VERTS[f][1]], p[FACE_VERTS[f][2]]);
            int32_t j = nbr[4 * i + f];
            if (j < 0) { dist[4 * i + f] = 0.0; g[4 * i + f] = 0.0; continue; }
            const double *q[4];
            for (int k = 0; k < 4; ++k) q[k] = verts + 3 * (int64_t)tets[4 * j + k];
            double cj[3];
            barycentre(q[0], q[1], q[2], q[3], cj);
            double dx = cj[0] - ci[0], dy = cj[1] - ci[1], dz = cj[2] - ci[2];
            dist[4 * i + f] = sqrt(dx * dx + dy * dy + dz * dz);
            g[4 * i + f] = area[4 * i + f] / (vol[i] * dist[4 * i + f]);
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t nt;
    int S, R;
    double D[ORC_MAXS];
    int lhs[ORC_MAXR][ORC_MAXS], rhs[ORC_MAXR][ORC_MAXS];
    double k[ORC_MAXR];
    int order[ORC_MAXR], ra[ORC_MAXR], rb[ORC_MAXR]; /* reactant species (-1 none) */
    int32_t *nbr;      /* [nt*4] */
    double *vol;       /* [nt] */
    double *g;         /* [nt*4] */
    double *cumg;      /* [nt*4] cumulative g over local faces */
    uint32_t *thr;     /* [nt*4] fixed-point cumulative thresholds at the full window */
    int leave_exp;     /* 1 = EXP leave law; thresholds from share and exp_leave() */
    uint32_t *share;   /* [nt*4] floor(2^31 cumg_f / G), EXP law only */
    double tau, dmax, gmax;
    int32_t *cnt;      /* [S*nt] current counts */
    int32_t *nxt;      /* [S*nt] */
    uint8_t *mask;     /* [R*nt] 1 = reaction active in tet (NULL row = all) */
    int has_mask[ORC_MAXR];
    uint64_t seed;
    int occ;           /* 1 = OCC (paper), 0 = END */
    int prec;          /* 64 = all FP64; 32 = reaction decisions in float like the kernel */
    double t_base;
    int64_t k_grid;
    uint64_t k_total;
    int64_t events;    /* reaction events fired so far */
    /* threaded (gather-form) windows only */
    int32_t *rev;      /* [nt*4] local face of the neighbour that points back, -1 on the boundary */
    int32_t *mv;       /* [S*nt*4] molecules tet i sends through face f, species-major */
} orc_sim;

/* tau from §2.1 and the fixed-point thresholds of every tet's faces. */
static void setup_rates(orc_sim *s)
{
    s->dmax = 0.0;
    for (int sp = 0; sp < s->S; ++sp) if (s->D[sp] > s->dmax) s->dmax = s->D[sp];
    s->gmax = 0.0;
    for (int64_t i = 0; i < s->nt; ++i) {
        double c = 0.0;
        for (int f = 0; f < 4; ++f) {
            c = c + s->g[4 * i + f];
            s->cumg[4 * i + f] = c;
        }
        if (c > s->gmax) s->gmax = c;
    }
    /* min over (S, tet) of 1/(D_S G_tet) == 1/(max D * max G): multiplication
     * is monotone, so the max of the products is the product of the maxima. */
    if (s->dmax > 0.0 && s->gmax > 0.0) s->tau = 1.0 / (s->dmax * s->gmax);
    else s->tau = INFINITY;
    /* A_{i,f} = floor(2^31 * tau*Dmax * cumg_{i,f}), clamped to [0, 2^31]. */
    double pt = isfinite(s->tau) ? s->tau * s->dmax : 0.0;
    for (int64_t i = 0; i < 4 * s->nt; ++i) {
        double x = (pt * s->cumg[i]) * 2147483648.0;
        double fl = floor(x);
        if (fl < 0.0) fl = 0.0;
        if (fl > 2147483648.0) fl = 2147483648.0;
        s->thr[i] = (uint32_t)fl;
    }
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->nbr); free(s->vol); free(s->g); free(s->cumg); free(s->thr); free(s->share);
    free(s->cnt); free(s->nxt); free(s->mask);
    free(s->rev); free(s->mv);
    free(s);
}

orc_sim *orc_create(int64_t nv, const double *verts, int64_t nt, const int32_t *tets,
                    int S, const double *D, int R, const int32_t *lhs, const int32_t *rhs,
                    const double *k, uint64_t seed, int occ, int prec, int *err)
{
    *err = ORC_OK;
    if (nt <= 0 || S <= 0 || S > ORC_MAXS || R < 0 || R > ORC_MAXR || (prec != 32 && prec != 64)) {
        *err = ORC_ERR_ARG;
        return NULL;
    }
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) { *err = ORC_ERR_OOM; return NULL; }
    s->nt = nt; s->S = S; s->R = R; s->seed = seed; s->occ = occ; s->prec = prec;
    for (int sp = 0; sp < S; ++sp) {
        if (!(D[sp] >= 0.0)) { *err = ORC_ERR_MODEL; orc_destroy(s); return NULL; }
        s->D[sp] = D[sp];
    }
    for (int r = 0; r < R; ++r) {
        int ord = 0, a = -1, b = -1;
        for (int sp = 0; sp < S; ++sp) {
            int l = lhs[r * S + sp], q = rhs[r * S + sp];
            if (l < 0 || q < 0) { *err = ORC_ERR_MODEL; orc_destroy(s); return NULL; }
            s->lhs[r][sp] = l; s->rhs[r][sp] = q;
            for (int m = 0; m < l; ++m) {
                if (a < 0) a = sp; else b = sp;
                ++ord;
            }
        }
        if (ord > 2 || !(k[r] >= 0.0)) { *err = ORC_ERR_MODEL; orc_destroy(s); return NULL; }
        s->order[r] = ord; s->ra[r] = a; s->rb[r] = b; s->k[r] = k[r];
    }
    s->nbr = (int32_t *)malloc(sizeof(int32_t) * 4 * nt);
    s->vol = (double *)malloc(sizeof(double) * nt);
    s->g = (double *)malloc(sizeof(double) * 4 * nt);
    s->cumg = (double *)malloc(sizeof(double) * 4 * nt);
    s->thr = (uint32_t *)malloc(sizeof(uint32_t) * 4 * nt);
    s->cnt = (int32_t *)calloc((size_t)S * nt, sizeof(int32_t));
    s->nxt = (int32_t *)calloc((size_t)S * nt, sizeof(int32_t));
    s->mask = (uint8_t *)calloc((size_t)(R > 0 ? R : 1) * nt, 1);
    double *area = (double *)malloc(sizeof(double) * 4 * nt);
    double *dist = (double *)malloc(sizeof(double) * 4 * nt);
    if (!s->nbr || !s->vol || !s->g || !s->cumg || !s->thr || !s->cnt || !s->nxt || !s->mask ||
        !area || !dist) {
        free(area); free(dist);
        *err = ORC_ERR_OOM; orc_destroy(s); return NULL;
    }
    int rc = orc_geometry(nv, verts, nt, tets, s->nbr, s->vol, area, dist, s->g);
    free(area); free(dist);
    if (rc) { *err = rc; orc_destroy(s); return NULL; }
    setup_rates(s);
    return s;
}

void orc_set_counts(orc_sim *s, int sp, const int32_t *c)
{
    memcpy(s->cnt + (size_t)sp * s->nt, c, sizeof(int32_t) * s->nt);
}

void orc_get_counts(const orc_sim *s, int sp, int32_t *out)
{
    memcpy(out, s->cnt + (size_t)sp * s->nt, sizeof(int32_t) * s->nt);
}

void orc_set_reac_mask(orc_sim *s, int r, const uint8_t *m)
{
    if (m) { memcpy(s->mask + (size_t)r * s->nt, m, s->nt); s->has_mask[r] = 1; }
    else s->has_mask[r] = 0;
}

/* Rate constant of reaction r from the next window on: the paper drives its
   calcium-burst runs with influx rates that change over time (§3.2). */
int orc_set_reac_rate(orc_sim *s, int r, double k)
{
    if (r < 0 || r >= s->R || !(k >= 0.0) || k != k || k - k != 0.0) return ORC_ERR_MODEL;
    s->k[r] = k;
    return 0;
}

double orc_get_tau(const orc_sim *s) { return s->tau; }
int64_t orc_get_events(const orc_sim *s) { return s->events; }
uint64_t orc_get_windows(const orc_sim *s) { return s->k_total; }

double orc_get_time(const orc_sim *s)
{
    return s->k_grid == 0 ? s->t_base : s->t_base + (double)s->k_grid * s->tau;
}

void orc_get_thresholds(const orc_sim *s, uint32_t *out) { memcpy(out, s->thr, sizeof(uint32_t) * 4 * s->nt); }
void orc_get_cumg(const orc_sim *s, double *out) { memcpy(out, s->cumg, sizeof(double) * 4 * s->nt); }

/* ------------------------------------------------------------------------ */
/* Reaction SSA operator for one tet over tau_k (Algorithm 1, reaction part). */
/* N holds the tet's counts on entry and the end-of-window counts on exit;   */
/* M receives the integer trial count of every species.                     */
/* ------------------------------------------------------------------------ */

/* Propensity in FP64: the plain mass-action definition. */
static double prop64(const orc_sim *s, int r, const int32_t *N, double nav)
{
    switch (s->order[r]) {
    case 0: return s->k[r] * nav;
    case 1: return s->k[r] * (double)N[s->ra[r]];
    default:
        if (s->ra[r] == s->rb[r])
            return s->k[r] / nav * (double)N[s->ra[r]] * (double)(N[s->ra[r]] - 1);
        return s->k[r] / nav * (double)N[s->ra[r]] * (double)N[s->rb[r]];
    }
}

/* Propensity with the kernel's float operations, in the kernel's order. */
static float prop32(const orc_sim *s, int r, const int32_t *N, float inv_nav)
{
    float kf = (float)s->k[r];
    switch (s->order[r]) {
    case 0: return kf / inv_nav;
    case 1: return kf * (float)N[s->ra[r]];
    default: {
        float c = kf * inv_nav;
        if (s->ra[r] == s->rb[r]) return (c * (float)N[s->ra[r]]) * (float)(N[s->ra[r]] - 1);
        return (c * (float)N[s->ra[r]]) * (float)N[s->rb[r]];
    }
    }
}

static void reaction_phase(const orc_sim *s, int64_t i, double tau_k, double inv_tau_k, int32_t *N, int32_t *M,
                           int64_t *events)
{
    double nav = ORC_AVOGADRO * (s->vol[i] * 1000.0); /* molecules per mol/L */
    float inv_nav = (float)(1.0 / nav);
    int active[ORC_MAXR];
    for (int r = 0; r < s->R; ++r) active[r] = !s->has_mask[r] || s->mask[(size_t)r * s->nt + i];

    double O[ORC_MAXS], tS[ORC_MAXS];
    int touched[ORC_MAXS];
    for (int sp = 0; sp < s->S; ++sp) { O[sp] = 0.0; tS[sp] = 0.0; touched[sp] = 0; }

    double dt_acc = 0.0; /* Delta t */
    uint32_t j = 0;       /* event draws so far in this window */
    for (;;) {
        int pick = -1;
        double dt_new;
        uint32_t w[4];
        if (s->prec == 64) {
            double a[ORC_MAXR], a0 = 0.0;
            for (int r = 0; r < s->R; ++r) { a[r] = active[r] ? prop64(s, r, N, nav) : 0.0; a0 += a[r]; }
            if (!(a0 > 0.0)) break;
            draw4(s->seed, s->k_total, (uint32_t)i, j++, ORC_PURPOSE_REAC, w);
            double dt = -log(unit53(w[0], w[1])) / a0;
            dt_new = dt_acc + dt;
            if (dt_new > tau_k) break;
            double target = unit53(w[2], w[3]) * a0, c = 0.0;
            for (int r = 0; r < s->R; ++r) {
                c += a[r];
                if (c > target) { pick = r; break; }
            }
            if (pick < 0) for (int r = s->R - 1; r >= 0; --r) if (a[r] > 0.0) { pick = r; break; }
        } else {
            float a[ORC_MAXR], a0 = 0.0f;
            for (int r = 0; r < s->R; ++r) { a[r] = active[r] ? prop32(s, r, N, inv_nav) : 0.0f; a0 = a0 + a[r]; }
            if (!(a0 > 0.0f)) break;
            draw4(s->seed, s->k_total, (uint32_t)i, j++, ORC_PURPOSE_REAC, w);
            float u1 = (float)unit24(w[0]);
            float dt = (-orc_logf32(u1)) / a0;
            dt_new = dt_acc + (double)dt;
            if (dt_new > tau_k) break;
            float target = (float)unit24(w[1]) * a0, c = 0.0f;
            for (int r = 0; r < s->R; ++r) {
                c = c + a[r];
                if (c > target) { pick = r; break; }
            }
            if (pick < 0) for (int r = s->R - 1; r >= 0; --r) if (a[r] > 0.0f) { pick = r; break; }
        }
        if (pick < 0) break; /* no next reaction */
        dt_acc = dt_new;
        /* occupancy of every species the reaction changes, then the change */
        for (int sp = 0; sp < s->S; ++sp) {
            int delta = s->rhs[pick][sp] - s->lhs[pick][sp];
            if (delta == 0) continue;
            O[sp] = O[sp] + (double)N[sp] * (dt_acc - tS[sp]);
            tS[sp] = dt_acc;
            touched[sp] = 1;
            N[sp] += delta;
        }
        (*events)++;
    }

    /* Mean occupancy -> integer trial count (Algorithm 1: Nbar = O_S / tau). */
    uint32_t rw[4];
    int have_block = -1;
    for (int sp = 0; sp < s->S; ++sp) {
        if (!s->occ || !touched[sp] || s->D[sp] <= 0.0) { M[sp] = N[sp]; continue; }
        double occ = O[sp] + (double)N[sp] * (tau_k - tS[sp]); /* close the integral at tau */
        double nbar = occ * inv_tau_k;
        double fl = floor(nbar);
        double frac = nbar - fl;
        if (have_block != sp / 4) {
            draw4(s->seed, s->k_total, (uint32_t)i, (uint32_t)(sp / 4), ORC_PURPOSE_ROUND, rw);
            have_block = sp / 4;
        }
        double u = ((double)rw[sp % 4] + 0.5) * (1.0 / 4294967296.0);
        int64_t m = (int64_t)fl + (u < frac ? 1 : 0);
        if (m < 0) m = 0;
        if (m > N[sp]) m = N[sp];
        M[sp] = (int32_t)m;
    }
}

/* One trial molecule per 31-bit word: face f if x < T_f (first such f), stay
 * if x >= T_3. Adds the number sent through each face to out[]. Returns the
 * number of words consumed (M, or 0 when nothing can leave). */
uint32_t orc_sample_faces(uint64_t seed, uint64_t window, uint32_t tet, uint32_t w0, int32_t M,
                          const uint32_t T[4], int32_t out[4])
{
    if (M <= 0 || T[3] == 0) return 0;
    uint32_t blk[4];
    uint32_t cur_block = 0xFFFFFFFFu;
    for (int32_t m = 0; m < M; ++m) {
        uint32_t w = w0 + (uint32_t)m;
        if ((w >> 2) != cur_block) {
            cur_block = w >> 2;
            draw4(seed, window, tet, cur_block, ORC_PURPOSE_DIFF, blk);
        }
        uint32_t x = blk[w & 3u] >> 1;
        for (int f = 0; f < 4; ++f) {
            if (x < T[f]) { out[f] += 1; break; }
        }
    }
    return (uint32_t)M;
}

/* The same decisions for a species with M >= ORC_BULK_MIN trial molecules:
 * molecule j of group g takes x = sum over planes k = 0..30 of
 * (bit j of plane k) << (30 - k), and goes through the first face f with
 * x < T_f (stays if x >= T_3). Adds the molecules sent through each face to
 * out[]. */
void orc_sample_bulk(uint64_t seed, uint64_t window, uint32_t tet, int sp, int32_t M, const uint32_t T[4],
                     int32_t out[4])
{
    if (M <= 0 || T[3] == 0) return;
    for (int64_t g = 0; 32 * g < (int64_t)M; ++g) {
        int m = (int64_t)M - 32 * g < 32 ? (int)((int64_t)M - 32 * g) : 32;
        uint32_t plane[32];
        for (uint32_t blk = 0; blk < 8; ++blk) draw4_bulk(seed, window, tet, sp, (uint32_t)g, blk, plane + 4 * blk);
        for (int j = 0; j < m; ++j) {
            uint32_t x = 0;
            for (int k = 0; k < 31; ++k) x |= ((plane[k] >> j) & 1u) << (30 - k);
            for (int f = 0; f < 4; ++f) {
                if (x < T[f]) { out[f] += 1; break; }
            }
        }
    }
}

/* The diffusion draws of species sp with M trial molecules in tet i: by bit
 * planes from ORC_BULK_MIN molecules on, else from the tet's word stream at
 * word *w (advanced past the words used). */
static void sample_species(const orc_sim *s, int64_t i, int sp, int32_t M, const uint32_t T[4], uint32_t *w,
                           int32_t leave[4])
{
    if (M >= ORC_BULK_MIN) orc_sample_bulk(s->seed, s->k_total, (uint32_t)i, sp, M, T, leave);
    else *w += orc_sample_faces(s->seed, s->k_total, (uint32_t)i, *w, M, T, leave);
}

/* Fixed-point species scale for a window of length tau_k:
 * R_S = floor(2^31 * (D_S / Dmax) * (tau_k / tau)), clamped to [0, 2^31]. */
static uint32_t species_scale(const orc_sim *s, int sp, double tau_k)
{
    if (!(s->D[sp] > 0.0) || !isfinite(s->tau)) return 0;
    double x = ((s->D[sp] / s->dmax) * (tau_k / s->tau)) * 2147483648.0;
    double fl = floor(x);
    if (fl < 0.0) fl = 0.0;
    if (fl > 2147483648.0) fl = 2147483648.0;
    return (uint32_t)fl;
}

/* EXP law: L = floor(2^31 (1 - exp(-(tau_k D_S) G_tet))), clamped to
 * [0, 2^31]; 0 for an immobile species. */
static uint32_t exp_leave(const orc_sim *s, int64_t i, int sp, double tau_k)
{
    if (!(s->D[sp] > 0.0) || !isfinite(s->tau)) return 0;
    double x = (tau_k * s->D[sp]) * s->cumg[4 * i + 3];
    double fl = floor((1.0 - exp(-x)) * 2147483648.0);
    if (fl < 0.0) fl = 0.0;
    if (fl > 2147483648.0) fl = 2147483648.0;
    return (uint32_t)fl;
}

/* Cumulative face thresholds of species sp in tet i for a window of length
 * tau_k whose species scale is `scale`: EULER T_f = (A_{i,f} * R_S) >> 31;
 * EXP T_f = (share_{i,f} * L_{S,i}) >> 31. */
static void species_thresholds(const orc_sim *s, int64_t i, int sp, double tau_k, uint32_t scale, uint32_t T[4])
{
    if (s->leave_exp) {
        uint32_t L = exp_leave(s, i, sp, tau_k);
        for (int f = 0; f < 4; ++f)
            T[f] = (uint32_t)(((uint64_t)s->share[4 * i + f] * (uint64_t)L) >> 31);
        return;
    }
    for (int f = 0; f < 4; ++f)
        T[f] = (uint32_t)(((uint64_t)s->thr[4 * i + f] * (uint64_t)scale) >> 31);
}

/* The thresholds every tet uses for species sp in a window of length tau_k
 * ([nt*4]), and the species scale R_S as the return value (EULER law). */
uint32_t orc_get_species_thresholds(const orc_sim *s, int sp, double tau_k, uint32_t *out)
{
    uint32_t scale = species_scale(s, sp, tau_k);
    for (int64_t i = 0; i < s->nt; ++i) species_thresholds(s, i, sp, tau_k, scale, out + 4 * i);
    return scale;
}

/* Leave law: 0 = EULER (p = tau d, default), 1 = EXP (p = 1 - exp(-tau d)). */
int orc_set_leave_law(orc_sim *s, int exp_law)
{
    if (exp_law != 0 && exp_law != 1) return ORC_ERR_ARG;
    if (exp_law && !s->share) {
        s->share = (uint32_t *)malloc(sizeof(uint32_t) * 4 * s->nt);
        if (!s->share) return ORC_ERR_OOM;
        for (int64_t i = 0; i < s->nt; ++i) {
            double G = s->cumg[4 * i + 3];
            for (int f = 0; f < 4; ++f) {
                double fl = G > 0.0 ? floor((s->cumg[4 * i + f] / G) * 2147483648.0) : 0.0;
                if (fl < 0.0) fl = 0.0;
                if (fl > 2147483648.0) fl = 2147483648.0;
                s->share[4 * i + f] = (uint32_t)fl;
            }
        }
    }
    s->leave_exp = exp_law;
    return ORC_OK;
}

/* One diffusion window of length tau_k over all tets (Algorithm 1). */
static void window(orc_sim *s, double tau_k)
{
    const int64_t nt = s->nt;
    const int S = s->S;
    double inv_tau_k = 1.0 / tau_k;
    uint32_t scale[ORC_MAXS];
    for (int sp = 0; sp < S; ++sp) scale[sp] = species_scale(s, sp, tau_k);
    memset(s->nxt, 0, sizeof(int32_t) * (size_t)S * nt);
    int32_t N[ORC_MAXS], M[ORC_MAXS];
    for (int64_t i = 0; i < nt; ++i) {
        for (int sp = 0; sp < S; ++sp) N[sp] = s->cnt[(size_t)sp * nt + i];
        /* reaction SSA operator */
        reaction_phase(s, i, tau_k, inv_tau_k, N, M, &s->events);
        /* diffusion operator: species in order; a species with few trial
         * molecules draws from the tet's word stream, one with many by bit planes */
        uint32_t w = 0;
        for (int sp = 0; sp < S; ++sp) {
            int32_t leave[4] = {0, 0, 0, 0};
            if (s->D[sp] > 0.0) {
                uint32_t T[4];
                species_thresholds(s, i, sp, tau_k, scale[sp], T);
                sample_species(s, i, sp, M[sp], T, &w, leave);
            }
            int32_t n = leave[0] + leave[1] + leave[2] + leave[3];
            s->nxt[(size_t)sp * nt + i] += N[sp] - n;
            for (int f = 0; f < 4; ++f)
                if (leave[f]) s->nxt[(size_t)sp * nt + s->nbr[4 * i + f]] += leave[f];
        }
    }
    int32_t *tmp = s->cnt; s->cnt = s->nxt; s->nxt = tmp;
    s->k_total++;
}

/* Advance to t_end (Algorithm 1 main loop). Time is t_base + k_grid * tau,
 * recomputed rather than accumulated. A full window is taken while
 * t + tau <= t_end (within 1e-9 tau); the last, shorter window uses a local
 * tau_k = t_end - t and leaves tau unchanged for later runs. */
int orc_run(orc_sim *s, double t_end)
{
    for (;;) {
        double t = orc_get_time(s);
        double tol = isfinite(s->tau) ? 1e-9 * s->tau : 0.0;
        if (!(t_end - t > tol)) break;
        if (isfinite(s->tau) && t + s->tau <= t_end + tol) {
            window(s, s->tau);
            s->k_grid++;
        } else {
            window(s, t_end - t);
            s->t_base = t_end;
            s->k_grid = 0;
            break;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* The same window on several host threads (the CPU baseline's all-core     */
/* figure). Jacobi in gather form: pass 1 runs every tet's reaction         */
/* operator and leave draws independently (each tet's draws depend only on  */
/* its own state and its own random stream) and records what it keeps and   */
/* what it sends through each face; pass 2 adds to every tet what its face   */
/* neighbours sent it. Integer sums, so the result is the serial window's,  */
/* bit for bit, whatever the thread count or schedule.                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    orc_sim *s;
    double tau_k, inv_tau_k;
    const uint32_t *scale;
    int pass;
    atomic_llong next;     /* next chunk of tets to take */
    atomic_llong events;
} orc_par_job;

enum { ORC_PAR_CHUNK = 256 };

static void par_tet_pass1(orc_par_job *job, int64_t i, int64_t *events)
{
    orc_sim *s = job->s;
    const int64_t nt = s->nt;
    int32_t N[ORC_MAXS], M[ORC_MAXS];
    for (int sp = 0; sp < s->S; ++sp) N[sp] = s->cnt[(size_t)sp * nt + i];
    reaction_phase(s, i, job->tau_k, job->inv_tau_k, N, M, events);
    uint32_t w = 0;
    for (int sp = 0; sp < s->S; ++sp) {
        int32_t leave[4] = {0, 0, 0, 0};
        if (s->D[sp] > 0.0) {
            uint32_t T[4];
            species_thresholds(s, i, sp, job->tau_k, job->scale[sp], T);
            sample_species(s, i, sp, M[sp], T, &w, leave);
        }
        int32_t n = leave[0] + leave[1] + leave[2] + leave[3];
        s->nxt[(size_t)sp * nt + i] = N[sp] - n;
        memcpy(s->mv + ((size_t)sp * nt + i) * 4, leave, sizeof(leave));
    }
}

static void par_tet_pass2(orc_sim *s, int64_t i)
{
    const int64_t nt = s->nt;
    for (int sp = 0; sp < s->S; ++sp) {
        int32_t add = 0;
        for (int f = 0; f < 4; ++f) {
            int32_t j = s->nbr[4 * i + f];
            if (j >= 0) add += s->mv[((size_t)sp * nt + j) * 4 + s->rev[4 * i + f]];
        }
        s->nxt[(size_t)sp * nt + i] += add;
    }
}

static void *par_worker(void *arg)
{
    orc_par_job *job = (orc_par_job *)arg;
    const int64_t nt = job->s->nt;
    int64_t events = 0;
    for (;;) {
        int64_t i0 = (int64_t)atomic_fetch_add(&job->next, ORC_PAR_CHUNK);
        if (i0 >= nt) break;
        int64_t i1 = i0 + ORC_PAR_CHUNK < nt ? i0 + ORC_PAR_CHUNK : nt;
        for (int64_t i = i0; i < i1; ++i) {
            if (job->pass == 1) par_tet_pass1(job, i, &events);
            else par_tet_pass2(job->s, i);
        }
    }
    atomic_fetch_add(&job->events, (long long)events);
    return NULL;
}

static int par_ensure(orc_sim *s)
{
    if (s->rev) return ORC_OK;
    s->rev = (int32_t *)malloc(sizeof(int32_t) * 4 * s->nt);
    s->mv = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)s->S * s->nt);
    if (!s->rev || !s->mv) { free(s->rev); free(s->mv); s->rev = s->mv = NULL; return ORC_ERR_OOM; }
    for (int64_t i = 0; i < s->nt; ++i)
        for (int f = 0; f < 4; ++f) {
            int32_t j = s->nbr[4 * i + f], back = -1;
            if (j >= 0)
                for (int g = 0; g < 4; ++g)
                    if (s->nbr[4 * (int64_t)j + g] == (int32_t)i) back = g;
            s->rev[4 * i + f] = back;
        }
    return ORC_OK;
}

static int par_pass(orc_par_job *job, int pass, int nthreads)
{
    pthread_t th[256];
    int started = 0;
    job->pass = pass;
    atomic_store(&job->next, 0);
    for (int k = 1; k < nthreads; ++k) {
        if (pthread_create(&th[started], NULL, par_worker, job) != 0) break;
        ++started;
    }
    par_worker(job); /* the calling thread works too */
    for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
    return ORC_OK;
}

static int window_threads(orc_sim *s, double tau_k, int nthreads)
{
    int rc = par_ensure(s);
    if (rc) return rc;
    uint32_t scale[ORC_MAXS];
    for (int sp = 0; sp < s->S; ++sp) scale[sp] = species_scale(s, sp, tau_k);
    orc_par_job job;
    job.s = s;
    job.tau_k = tau_k;
    job.inv_tau_k = 1.0 / tau_k;
    job.scale = scale;
    atomic_init(&job.next, 0);
    atomic_init(&job.events, 0);
    par_pass(&job, 1, nthreads);
    par_pass(&job, 2, nthreads);
    s->events += (int64_t)atomic_load(&job.events);
    int32_t *tmp = s->cnt; s->cnt = s->nxt; s->nxt = tmp;
    s->k_total++;
    return ORC_OK;
}

/* orc_run on `nthreads` host threads (1..256): the same windows, the same result. */
int orc_run_threads(orc_sim *s, double t_end, int nthreads)
{
    if (nthreads < 1 || nthreads > 256) return ORC_ERR_ARG;
    for (;;) {
        double t = orc_get_time(s);
        double tol = isfinite(s->tau) ? 1e-9 * s->tau : 0.0;
        if (!(t_end - t > tol)) break;
        int rc;
        if (isfinite(s->tau) && t + s->tau <= t_end + tol) {
            rc = window_threads(s, s->tau, nthreads);
            if (rc) return rc;
            s->k_grid++;
        } else {
            rc = window_threads(s, t_end - t, nthreads);
            if (rc) return rc;
            s->t_base = t_end;
            s->k_grid = 0;
            break;
        }
    }
    return ORC_OK;
}

/* One window of explicit length on `nthreads` host threads. */
int orc_step_threads(orc_sim *s, double tau_k, int nthreads)
{
    if (nthreads < 1 || nthreads > 256) return ORC_ERR_ARG;
    return window_threads(s, tau_k, nthreads);
}

/* One window of explicit length (for tests of the operator on its own). */
int orc_step(orc_sim *s, double tau_k)
{
    window(s, tau_k);
    return ORC_OK;
}

/* Array forms of the building blocks, for exhaustive comparisons. */
void orc_logf32_array(const float *x, int64_t n, float *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_logf32(x[i]);
}

void orc_philox_array(uint64_t seed, const uint32_t *ctr, int64_t n, uint32_t *out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(key, ctr + 4 * i, out + 4 * i);
}
