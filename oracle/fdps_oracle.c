/*
 * fdps_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the Barnes-Hut long-range force of
 * FDPS (Iwasawa et al. 2016, arXiv 1601.03138) for softened self-gravity.
 * It exists to check the CUDA path; only the test suite, the package's smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header or constant with the CUDA library.
 *
 * What it computes, step by step, in the order of the paper's Sect. 3.2
 * (build a tree of the particles, then traverse it per group of i-particles
 * with a fixed opening angle):
 *   root box -> Morton keys -> stable sort -> octree (BFS order) ->
 *   moments (monopole, traceless quadrupole) -> i-groups (Barnes 1990,
 *   Sect. 5.5, eq. wtime_force) -> per-group walk with a fixed opening angle
 *   -> forces from the lists (Eqs. ParticleParticleNbody and
 *   ParticleSuperparticleNbody, Sect. 2.2) -> leapfrog kick/drift (Sect. 2.2,
 *   the predict/correct member functions of the N-body example).
 * Plus the exact reference: an O(N^2) FP64 direct sum of the same softened
 * pair force; and the short-range mode's brute-force neighbour counts and
 * SPH density (Wendland C6) for the paper's four cutoff types.
 *
 * The paper fixes the force law and the Barnes-Hut structure but not the key
 * scheme, the tree rules, the opening criterion, the quadrupole convention,
 * group selection or the potential.  The readings taken here are:
 *   keys   : q_a = min(2^21-1, floor((x_a - lo_a) * s)), s = 2^21 / L,
 *            L = largest box extent (1 if 0); key bit 3b+2/3b+1/3b = bit b
 *            of q_x/q_y/q_z (63-bit Morton key).
 *   sort   : stable by key (ties keep input order).
 *   tree   : node = (level l, key prefix) with at least one particle; a
 *            node is a leaf iff count <= n_leaf or l = 21; children are the
 *            non-empty octants in digit order; node ids in BFS order
 *            (level-major, prefix ascending).
 *   moments: M and S = sum m x summed sequentially (leaves: over particles in
 *            sorted order; internal nodes: over children in octant order),
 *            COM = S / M (0 if M = 0); traceless quadrupole about the COM,
 *            Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab), from the particles.
 *   groups : depth-first from the root; a node with count <= n_grp, or a
 *            leaf, is a group and is not descended.
 *   opening: open cell C for group G iff C's grid cube meets G's grid box
 *            (closed integer intervals of quantised coordinates), or
 *            ell_C^2 >= theta^2 d^2, with ell_C = L 2^-l and d the distance
 *            from C's COM to G's FP64 bounding box.  Opened leaf -> its
 *            particles go to the EPJ list; unopened cell -> SPJ list.
 *   force  : acceleration of Eq. ParticleParticleNbody with the
 *            i-particle's softening; potential -sum m/sqrt(r^2+eps_i^2)
 *            with the self term removed (+ m_i/eps_i); quadrupole
 *            superparticle: phi = -M/R - (r.Q.r)/(2R^5) with
 *            R^2 = r^2 + eps_i^2 and a = -grad phi.
 * Compiled with -ffp-contract=off: every FP64 product and sum is rounded on
 * its own, so the root box, keys, centres of mass and opening decisions are
 * reproducible bit for bit by any implementation that performs the same
 * operations in the same order.
 */
#include "fdps_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXLEVEL 21
#define ORC_QMAX 2097151ULL /* 2^21 - 1 */

typedef struct {
    int32_t level;
    uint64_t prefix;
    int64_t first, count;
    int64_t child_first; /* -1 for a leaf */
    int32_t nchild;
    int32_t is_leaf;
    uint32_t qlo[3];
    double mass, sum[3], com[3], quad[6]; /* quad: xx yy zz xy xz yz */
} orc_node;

typedef struct {
    int64_t first, count, node;
    double lo[3], hi[3];
    uint32_t qmin[3], qmax[3];
} orc_group;

struct orc_tree {
    int64_t n;
    int32_t n_leaf, n_grp, quad;
    double theta, theta2;
    double lo[3], L, s;
    uint64_t* keys_in;  /* keys in input order */
    uint32_t* perm;     /* sorted position -> input index */
    uint64_t* keys;     /* sorted keys */
    double* pos;        /* sorted positions [n][3] */
    double* mass;       /* sorted */
    double* eps;        /* sorted */
    uint32_t* q;        /* sorted quantised coordinates [n][3] */
    orc_node* nodes;
    int64_t n_nodes, cap_nodes;
    orc_group* groups;
    int64_t n_groups, cap_groups;
};

/* ---------------------------------------------------------------- O1 box */

int orc_root_box(int64_t n, const double* pos, double* lo3, double* L_out,
                 double* s_out) {
    if (n <= 0) return -1;
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = pos[a];
    for (int64_t i = 1; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = pos[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    double L = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = hi[a] - lo[a];
        if (e > L) L = e;
    }
    if (L == 0.0) L = 1.0;
    for (int a = 0; a < 3; ++a) lo3[a] = lo[a];
    *L_out = L;
    *s_out = 2097152.0 / L; /* 2^21 / L, one rounded divide */
    return 0;
}

/* ---------------------------------------------------------------- O2 keys */

static uint32_t orc_quantise(double x, double lo, double s) {
    double t = x - lo;
    double u = t * s;
    double f = floor(u);
    if (f > (double)ORC_QMAX) f = (double)ORC_QMAX;
    if (f < 0.0) f = 0.0;
    return (uint32_t)f;
}

uint64_t orc_morton(uint32_t qx, uint32_t qy, uint32_t qz) {
    uint64_t key = 0;
    for (int b = 0; b < ORC_MAXLEVEL; ++b) {
        key |= (uint64_t)((qx >> b) & 1u) << (3 * b + 2);
        key |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);
        key |= (uint64_t)((qz >> b) & 1u) << (3 * b);
    }
    return key;
}

void orc_keys(int64_t n, const double* pos, const double* lo3, double s,
              uint64_t* keys, uint32_t* q3) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) q[a] = orc_quantise(pos[3 * i + a], lo3[a], s);
        keys[i] = orc_morton(q[0], q[1], q[2]);
        if (q3)
            for (int a = 0; a < 3; ++a) q3[3 * i + a] = q[a];
    }
}

/* ---------------------------------------------------------------- O3 sort */

typedef struct {
    uint64_t key;
    uint32_t idx;
} orc_kv;

static int orc_kv_cmp(const void* pa, const void* pb) {
    const orc_kv* a = (const orc_kv*)pa;
    const orc_kv* b = (const orc_kv*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

/* Ordering by (key, input index) is the stable order by key. */
void orc_sort(int64_t n, const uint64_t* keys, uint32_t* perm) {
    orc_kv* kv = (orc_kv*)malloc(sizeof(orc_kv) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        kv[i].key = keys[i];
        kv[i].idx = (uint32_t)i;
    }
    qsort(kv, (size_t)n, sizeof(orc_kv), orc_kv_cmp);
    for (int64_t i = 0; i < n; ++i) perm[i] = kv[i].idx;
    free(kv);
}

/* --------------------------------------------------------------- O4 tree */

static int64_t orc_push_node(orc_tree* t) {
    if (t->n_nodes == t->cap_nodes) {
        t->cap_nodes = t->cap_nodes ? 2 * t->cap_nodes : 1024;
        t->nodes = (orc_node*)realloc(t->nodes, sizeof(orc_node) * (size_t)t->cap_nodes);
    }
    memset(&t->nodes[t->n_nodes], 0, sizeof(orc_node));
    return t->n_nodes++;
}

static void orc_cell_origin(int32_t level, uint64_t prefix, uint32_t qlo[3]) {
    uint32_t p[3] = {0, 0, 0};
    for (int k = 0; k < level; ++k) {
        p[0] |= (uint32_t)((prefix >> (3 * k + 2)) & 1u) << k;
        p[1] |= (uint32_t)((prefix >> (3 * k + 1)) & 1u) << k;
        p[2] |= (uint32_t)((prefix >> (3 * k)) & 1u) << k;
    }
    for (int a = 0; a < 3; ++a) qlo[a] = p[a] << (ORC_MAXLEVEL - level);
}

static void orc_build_nodes(orc_tree* t) {
    int64_t r = orc_push_node(t);
    t->nodes[r].level = 0;
    t->nodes[r].prefix = 0;
    t->nodes[r].first = 0;
    t->nodes[r].count = t->n;
    /* Nodes are appended while the array is scanned front to back, so the
       array is its own FIFO queue and ids come out in BFS order. */
    for (int64_t id = 0; id < t->n_nodes; ++id) {
        orc_node nd = t->nodes[id];
        orc_cell_origin(nd.level, nd.prefix, t->nodes[id].qlo);
        if (nd.count <= t->n_leaf || nd.level == ORC_MAXLEVEL) {
            t->nodes[id].is_leaf = 1;
            t->nodes[id].child_first = -1;
            t->nodes[id].nchild = 0;
            continue;
        }
        int32_t cl = nd.level + 1;
        int shift = 63 - 3 * cl;
        int64_t i = nd.first, end = nd.first + nd.count;
        int64_t first_child = -1;
        int32_t nc = 0;
        while (i < end) {
            uint64_t digit = (t->keys[i] >> shift) & 7u;
            int64_t j = i;
            while (j < end && ((t->keys[j] >> shift) & 7u) == digit) ++j;
            int64_t c = orc_push_node(t);
            if (first_child < 0) first_child = c;
            t->nodes[c].level = cl;
            t->nodes[c].prefix = (nd.prefix << 3) | digit;
            t->nodes[c].first = i;
            t->nodes[c].count = j - i;
            ++nc;
            i = j;
        }
        t->nodes[id].is_leaf = 0;
        t->nodes[id].child_first = first_child;
        t->nodes[id].nchild = nc;
    }
}

/* ------------------------------------------- multipole helpers (O5, O10) */

/* Traceless quadrupole about c: Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab),
   d = x - c, summed over the particles in their order.  Q = {xx,yy,zz,xy,xz,yz}. */
void orc_quadrupole(int64_t n, const double* pos, const double* mass,
                    const double* c, double* Q) {
    for (int k = 0; k < 6; ++k) Q[k] = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        double m = mass[p];
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = pos[3 * p + a] - c[a];
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        Q[0] += m * (3.0 * d[0] * d[0] - d2);
        Q[1] += m * (3.0 * d[1] * d[1] - d2);
        Q[2] += m * (3.0 * d[2] * d[2] - d2);
        Q[3] += m * (3.0 * d[0] * d[1]);
        Q[4] += m * (3.0 * d[0] * d[2]);
        Q[5] += m * (3.0 * d[1] * d[2]);
    }
}

/* Monopole and quadrupole of a particle set: M, COM = sum m x / M, Q about COM. */
void orc_multipole(int64_t n, const double* pos, const double* mass,
                   double* M_out, double* com, double* Q) {
    double M = 0.0, S[3] = {0.0, 0.0, 0.0};
    for (int64_t p = 0; p < n; ++p) {
        M = M + mass[p];
        for (int a = 0; a < 3; ++a) {
            double mx = mass[p] * pos[3 * p + a];
            S[a] = S[a] + mx;
        }
    }
    for (int a = 0; a < 3; ++a) com[a] = (M > 0.0) ? S[a] / M : 0.0;
    *M_out = M;
    orc_quadrupole(n, pos, mass, com, Q);
}

/* Interaction of one superparticle (mass M at com, traceless quadrupole Q
   when Q != NULL) with a particle at xi softened by eps_i (ep2 = eps_i^2):
   adds -grad phi to acc3 and phi to pot, where r = xi - com,
   R^2 = |r|^2 + ep2 and phi = -M/R - (r.Q.r) / (2 R^5). */
void orc_spj_force(const double* xi, double ep2, double M, const double* com,
                   const double* Q, double* acc3, double* pot) {
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = xi[a] - com[a];
    double R2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + ep2;
    double Rinv = 1.0 / sqrt(R2);
    double Rinv2 = Rinv * Rinv;
    double Rinv3 = Rinv2 * Rinv;
    for (int a = 0; a < 3; ++a) acc3[a] -= M * Rinv3 * r[a];
    *pot -= M * Rinv;
    if (Q) {
        double Qr[3];
        Qr[0] = Q[0] * r[0] + Q[3] * r[1] + Q[4] * r[2];
        Qr[1] = Q[3] * r[0] + Q[1] * r[1] + Q[5] * r[2];
        Qr[2] = Q[4] * r[0] + Q[5] * r[1] + Q[2] * r[2];
        double rQr = r[0] * Qr[0] + r[1] * Qr[1] + r[2] * Qr[2];
        double Rinv5 = Rinv3 * Rinv2;
        double Rinv7 = Rinv5 * Rinv2;
        for (int a = 0; a < 3; ++a) acc3[a] += Qr[a] * Rinv5 - 2.5 * rQr * Rinv7 * r[a];
        *pot -= 0.5 * rQr * Rinv5;
    }
}

/* ------------------------------------------------------------ O5 moments */

static void orc_moments(orc_tree* t) {
    /* Children carry larger ids than their parent (BFS), so a reverse scan
       visits every child before its parent. */
    for (int64_t id = t->n_nodes - 1; id >= 0; --id) {
        orc_node* nd = &t->nodes[id];
        double M = 0.0, S[3] = {0.0, 0.0, 0.0};
        if (nd->is_leaf) {
            for (int64_t p = nd->first; p < nd->first + nd->count; ++p) {
                double m = t->mass[p];
                M = M + m;
                for (int a = 0; a < 3; ++a) {
                    double mx = m * t->pos[3 * p + a];
                    S[a] = S[a] + mx;
                }
            }
        } else {
            for (int32_t c = 0; c < nd->nchild; ++c) {
                const orc_node* ch = &t->nodes[nd->child_first + c];
                M = M + ch->mass;
                for (int a = 0; a < 3; ++a) S[a] = S[a] + ch->sum[a];
            }
        }
        nd->mass = M;
        for (int a = 0; a < 3; ++a) {
            nd->sum[a] = S[a];
            nd->com[a] = (M > 0.0) ? S[a] / M : 0.0;
        }
    }
    if (!t->quad) return;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t id = 0; id < t->n_nodes; ++id) {
        orc_node* nd = &t->nodes[id];
        orc_quadrupole(nd->count, &t->pos[3 * nd->first], &t->mass[nd->first],
                       nd->com, nd->quad);
    }
}

/* ------------------------------------------------------------- O6 groups */

static void orc_push_group(orc_tree* t, int64_t node) {
    if (t->n_groups == t->cap_groups) {
        t->cap_groups = t->cap_groups ? 2 * t->cap_groups : 1024;
        t->groups = (orc_group*)realloc(t->groups, sizeof(orc_group) * (size_t)t->cap_groups);
    }
    orc_group* g = &t->groups[t->n_groups++];
    const orc_node* nd = &t->nodes[node];
    g->first = nd->first;
    g->count = nd->count;
    g->node = node;
    for (int a = 0; a < 3; ++a) {
        g->lo[a] = g->hi[a] = t->pos[3 * nd->first + a];
        g->qmin[a] = g->qmax[a] = t->q[3 * nd->first + a];
    }
    for (int64_t p = nd->first; p < nd->first + nd->count; ++p)
        for (int a = 0; a < 3; ++a) {
            double v = t->pos[3 * p + a];
            uint32_t qa = t->q[3 * p + a];
            if (v < g->lo[a]) g->lo[a] = v;
            if (v > g->hi[a]) g->hi[a] = v;
            if (qa < g->qmin[a]) g->qmin[a] = qa;
            if (qa > g->qmax[a]) g->qmax[a] = qa;
        }
}

static void orc_groups_dfs(orc_tree* t, int64_t node) {
    const orc_node* nd = &t->nodes[node];
    if (nd->count <= t->n_grp || nd->is_leaf) {
        orc_push_group(t, node);
        return;
    }
    for (int32_t c = 0; c < nd->nchild; ++c) orc_groups_dfs(t, nd->child_first + c);
}

/* ------------------------------------------------------ O7/O8 the walk */

int orc_open_cell(const orc_tree* t, int64_t node, int64_t group) {
    const orc_node* c = &t->nodes[node];
    const orc_group* g = &t->groups[group];
    uint32_t w = (uint32_t)((1u << (ORC_MAXLEVEL - c->level)) - 1u);
    int meets = 1;
    for (int a = 0; a < 3; ++a)
        if (c->qlo[a] > g->qmax[a] || c->qlo[a] + w < g->qmin[a]) meets = 0;
    if (meets) return 1;
    double ell = ldexp(t->L, -c->level);
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double below = g->lo[a] - c->com[a];
        double above = c->com[a] - g->hi[a];
        double da = below > 0.0 ? below : (above > 0.0 ? above : 0.0);
        double sq = da * da;
        d2 = d2 + sq;
    }
    double lhs = ell * ell;
    double rhs = t->theta2 * d2;
    return lhs >= rhs;
}

typedef struct {
    int64_t *epj, n_epj, cap_epj;
    int64_t *spj, n_spj, cap_spj;
    int overflow;
} orc_list;

static void orc_list_add(int64_t** arr, int64_t* n, int64_t* cap, int64_t v,
                         int growable, int* overflow) {
    if (*n == *cap) {
        if (!growable) {
            *overflow = 1;
            ++*n;
            return;
        }
        *cap = *cap ? 2 * *cap : 256;
        *arr = (int64_t*)realloc(*arr, sizeof(int64_t) * (size_t)*cap);
    }
    (*arr)[(*n)++] = v;
}

static void orc_walk_dfs(const orc_tree* t, int64_t node, int64_t group,
                         orc_list* L, int growable) {
    const orc_node* c = &t->nodes[node];
    if (!orc_open_cell(t, node, group)) {
        orc_list_add(&L->spj, &L->n_spj, &L->cap_spj, node, growable, &L->overflow);
        return;
    }
    if (c->is_leaf) {
        for (int64_t p = c->first; p < c->first + c->count; ++p)
            orc_list_add(&L->epj, &L->n_epj, &L->cap_epj, p, growable, &L->overflow);
        return;
    }
    for (int32_t k = 0; k < c->nchild; ++k)
        orc_walk_dfs(t, c->child_first + k, group, L, growable);
}

int64_t orc_tree_walk(const orc_tree* t, int64_t group, int64_t* epj,
                      int64_t cap_epj, int64_t* n_epj, int64_t* spj,
                      int64_t cap_spj, int64_t* n_spj) {
    if (group < 0 || group >= t->n_groups) return -1;
    orc_list L = {epj, 0, cap_epj, spj, 0, cap_spj, 0};
    orc_walk_dfs(t, 0, group, &L, 0);
    *n_epj = L.n_epj;
    *n_spj = L.n_spj;
    return L.overflow ? 1 : 0;
}

/* ------------------------------------------------------------- O10 force */

static void orc_force_group(const orc_tree* t, int64_t group, const orc_list* L,
                            double* acc_sorted, double* pot_sorted) {
    const orc_group* g = &t->groups[group];
    for (int64_t i = g->first; i < g->first + g->count; ++i) {
        const double* xi = &t->pos[3 * i];
        double ep2 = t->eps[i] * t->eps[i];
        double ai[3] = {0.0, 0.0, 0.0};
        double phi = 0.0;
        /* particle-particle, Eq. ParticleParticleNbody */
        for (int64_t k = 0; k < L->n_epj; ++k) {
            int64_t j = L->epj[k];
            double dr[3];
            for (int a = 0; a < 3; ++a) dr[a] = xi[a] - t->pos[3 * j + a];
            double r2 = dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2] + ep2;
            double rinv = 1.0 / sqrt(r2);
            double mr3 = t->mass[j] * rinv * rinv * rinv;
            for (int a = 0; a < 3; ++a) ai[a] -= mr3 * dr[a];
            phi -= t->mass[j] * rinv;
        }
        /* particle-superparticle, Eq. ParticleSuperparticleNbody */
        for (int64_t k = 0; k < L->n_spj; ++k) {
            const orc_node* c = &t->nodes[L->spj[k]];
            orc_spj_force(xi, ep2, c->mass, c->com, t->quad ? c->quad : NULL, ai, &phi);
        }
        /* The list holds the i-particle itself: its force term is zero
           (dr = 0) and its potential term -m_i/eps_i is removed here. */
        phi += t->mass[i] / t->eps[i];
        for (int a = 0; a < 3; ++a) acc_sorted[3 * i + a] = ai[a];
        pot_sorted[i] = phi;
    }
}

/* ------------------------------------------------------------- the tree */

orc_tree* orc_tree_build(int64_t n, const double* pos, const double* mass,
                         const double* eps, double theta, int32_t n_leaf,
                         int32_t n_grp, int32_t quad) {
    if (n <= 0 || n > 0xFFFFFFFFLL || theta < 0.0 || n_leaf < 1 || n_grp < n_leaf)
        return NULL;
    orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
    t->n = n;
    t->n_leaf = n_leaf;
    t->n_grp = n_grp;
    t->quad = quad ? 1 : 0;
    t->theta = theta;
    t->theta2 = theta * theta;
    orc_root_box(n, pos, t->lo, &t->L, &t->s);
    t->keys_in = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    uint32_t* q_in = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    orc_keys(n, pos, t->lo, t->s, t->keys_in, q_in);
    t->perm = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    orc_sort(n, t->keys_in, t->perm);
    t->keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    t->pos = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    t->mass = (double*)malloc(sizeof(double) * (size_t)n);
    t->eps = (double*)malloc(sizeof(double) * (size_t)n);
    t->q = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t src = t->perm[i];
        t->keys[i] = t->keys_in[src];
        for (int a = 0; a < 3; ++a) {
            t->pos[3 * i + a] = pos[3 * (int64_t)src + a];
            t->q[3 * i + a] = q_in[3 * (int64_t)src + a];
        }
        t->mass[i] = mass[src];
        t->eps[i] = eps[src];
    }
    free(q_in);
    orc_build_nodes(t);
    orc_moments(t);
    orc_groups_dfs(t, 0);
    return t;
}

void orc_tree_free(orc_tree* t) {
    if (!t) return;
    free(t->keys_in);
    free(t->perm);
    free(t->keys);
    free(t->pos);
    free(t->mass);
    free(t->eps);
    free(t->q);
    free(t->nodes);
    free(t->groups);
    free(t);
}

int64_t orc_tree_n_nodes(const orc_tree* t) { return t->n_nodes; }
int64_t orc_tree_n_groups(const orc_tree* t) { return t->n_groups; }

void orc_tree_box(const orc_tree* t, double* out5) {
    for (int a = 0; a < 3; ++a) out5[a] = t->lo[a];
    out5[3] = t->L;
    out5[4] = t->s;
}

void orc_tree_keys(const orc_tree* t, uint64_t* keys_in, uint32_t* perm) {
    memcpy(keys_in, t->keys_in, sizeof(uint64_t) * (size_t)t->n);
    memcpy(perm, t->perm, sizeof(uint32_t) * (size_t)t->n);
}

void orc_tree_nodes(const orc_tree* t, int32_t* level, uint64_t* prefix,
                    int64_t* first, int64_t* count, int64_t* child_first,
                    int32_t* nchild, double* mass, double* com, double* quad) {
    for (int64_t i = 0; i < t->n_nodes; ++i) {
        const orc_node* nd = &t->nodes[i];
        if (level) level[i] = nd->level;
        if (prefix) prefix[i] = nd->prefix;
        if (first) first[i] = nd->first;
        if (count) count[i] = nd->count;
        if (child_first) child_first[i] = nd->child_first;
        if (nchild) nchild[i] = nd->nchild;
        if (mass) mass[i] = nd->mass;
        for (int a = 0; a < 3; ++a)
            if (com) com[3 * i + a] = nd->com[a];
        for (int k = 0; k < 6; ++k)
            if (quad) quad[6 * i + k] = nd->quad[k];
    }
}

void orc_tree_groups(const orc_tree* t, int64_t* first, int64_t* count,
                     int64_t* node, double* box6, uint32_t* qbox6) {
    for (int64_t g = 0; g < t->n_groups; ++g) {
        const orc_group* gr = &t->groups[g];
        if (first) first[g] = gr->first;
        if (count) count[g] = gr->count;
        if (node) node[g] = gr->node;
        for (int a = 0; a < 3; ++a) {
            if (box6) {
                box6[6 * g + a] = gr->lo[a];
                box6[6 * g + 3 + a] = gr->hi[a];
            }
            if (qbox6) {
                qbox6[6 * g + a] = gr->qmin[a];
                qbox6[6 * g + 3 + a] = gr->qmax[a];
            }
        }
    }
}

/* Forces for the particles of the listed groups (all groups if gidx is NULL).
   Results are written in INPUT order; rows of particles outside the listed
   groups are left untouched.  totals (may be NULL) receives
   {sum |EPJ|, sum |SPJ|, sum n_i (|EPJ| + |SPJ|), sum n_i |SPJ|}. */
void orc_tree_force(const orc_tree* t, const int64_t* gidx, int64_t ng,
                    double* acc_in, double* pot_in, int64_t* totals) {
    int64_t ngroups = gidx ? ng : t->n_groups;
    int64_t tot_e = 0, tot_s = 0, tot_int = 0, tot_spi = 0;
    double* acc_s = (double*)malloc(sizeof(double) * 3 * (size_t)t->n);
    double* pot_s = (double*)malloc(sizeof(double) * (size_t)t->n);
#pragma omp parallel reduction(+ : tot_e, tot_s, tot_int, tot_spi)
    {
        orc_list L = {NULL, 0, 0, NULL, 0, 0, 0};
#pragma omp for schedule(dynamic, 1)
        for (int64_t k = 0; k < ngroups; ++k) {
            int64_t g = gidx ? gidx[k] : k;
            L.n_epj = L.n_spj = 0;
            orc_walk_dfs(t, 0, g, &L, 1);
            orc_force_group(t, g, &L, acc_s, pot_s);
            int64_t ni = t->groups[g].count;
            tot_e += L.n_epj;
            tot_s += L.n_spj;
            tot_int += ni * (L.n_epj + L.n_spj);
            tot_spi += ni * L.n_spj;
        }
        free(L.epj);
        free(L.spj);
    }
    for (int64_t k = 0; k < ngroups; ++k) {
        const orc_group* g = &t->groups[gidx ? gidx[k] : k];
        for (int64_t i = g->first; i < g->first + g->count; ++i) {
            int64_t dst = t->perm[i];
            for (int a = 0; a < 3; ++a) acc_in[3 * dst + a] = acc_s[3 * i + a];
            pot_in[dst] = pot_s[i];
        }
    }
    free(acc_s);
    free(pot_s);
    if (totals) {
        totals[0] = tot_e;
        totals[1] = tot_s;
        totals[2] = tot_int;
        totals[3] = tot_spi;
    }
}

/* ------------------------------------------------------ O11 direct sum */

/* Exact reference: for each listed i (all if idx is NULL), the FP64 sum over
   j != i in index order of Eq. ParticleParticleNbody with eps_i, and the
   potential -sum_{j != i} m_j / sqrt(r^2 + eps_i^2).  Row k of acc/pot
   belongs to particle idx[k] (to particle k if idx is NULL). */
void orc_direct(int64_t n, const double* pos, const double* mass,
                const double* eps, const int64_t* idx, int64_t ni,
                double* acc, double* pot) {
    int64_t m_i = idx ? ni : n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < m_i; ++k) {
        int64_t i = idx ? idx[k] : k;
        double ep2 = eps[i] * eps[i];
        double ai[3] = {0.0, 0.0, 0.0};
        double phi = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dr[3];
            for (int a = 0; a < 3; ++a) dr[a] = pos[3 * j + a] - pos[3 * i + a];
            double r2 = dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2] + ep2;
            double rinv = 1.0 / sqrt(r2);
            double mr3 = mass[j] * rinv * rinv * rinv;
            for (int a = 0; a < 3; ++a) ai[a] += mr3 * dr[a];
            phi -= mass[j] * rinv;
        }
        for (int a = 0; a < 3; ++a) acc[3 * k + a] = ai[a];
        pot[k] = phi;
    }
}

/* ------------------------------------------------- short-range mode (S) */
/*
 * The short-range interaction (Sect. 2.1.2, 3.2): particle j is a neighbour
 * of particle i (j = i included, at zero separation) iff r^2 < c^2, with
 * r^2 = (dx*dx + dy*dy) + dz*dz, dx = x_j - x_i, each operation rounded on
 * its own, and the cutoff c of the paper's four types:
 *   mode 0 fixed:        c = r_fixed
 *   mode 1 i-dependent:  c = h_i         (gather)
 *   mode 2 j-dependent:  c = h_j         (scatter)
 *   mode 3 symmetric:    c = max(h_i, h_j)
 * The workload on the neighbours is the SPH density with the Wendland C6
 * kernel the paper uses for its SPH runs (Sect. 4.3): rho_i = sum_j m_j
 * W(r, H) with H = r_fixed, h_i, h_j respectively, and for the symmetric
 * type the mean of W(r, h_i) and W(r, h_j).  Brute force over all pairs.
 */
double orc_wendland_c6(double r, double H) {
    if (!(H > 0.0)) return 0.0;
    double q = r / H;
    if (q >= 1.0) return 0.0;
    double u = 1.0 - q, u2 = u * u, u4 = u2 * u2, u8 = u4 * u4;
    double poly = 1.0 + q * (8.0 + q * (25.0 + q * 32.0));
    const double pi = 3.14159265358979323846;
    return 1365.0 / (64.0 * pi * H * H * H) * u8 * poly;
}

void orc_wendland_c6_array(int64_t n, const double* r, double H, double* out) {
    for (int64_t k = 0; k < n; ++k) out[k] = orc_wendland_c6(r[k], H);
}

void orc_neighbors(int64_t n, const double* pos, const double* mass, const double* h,
                   int32_t mode, double r_fixed, const int64_t* idx, int64_t ni,
                   int64_t* count, double* rho) {
    int64_t m_i = idx ? ni : n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < m_i; ++k) {
        int64_t i = idx ? idx[k] : k;
        int64_t cnt = 0;
        double sum = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double dx = pos[3 * j] - pos[3 * i];
            double dy = pos[3 * j + 1] - pos[3 * i + 1];
            double dz = pos[3 * j + 2] - pos[3 * i + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double c = mode == 0 ? r_fixed : mode == 1 ? h[i] : mode == 2 ? h[j] : (h[i] > h[j] ? h[i] : h[j]);
            if (!(r2 < c * c)) continue;
            ++cnt;
            double r = sqrt(r2);
            double w = mode == 0 ? orc_wendland_c6(r, r_fixed)
                     : mode == 1 ? orc_wendland_c6(r, h[i])
                     : mode == 2 ? orc_wendland_c6(r, h[j])
                                 : 0.5 * (orc_wendland_c6(r, h[i]) + orc_wendland_c6(r, h[j]));
            sum += mass[j] * w;
        }
        count[k] = cnt;
        rho[k] = sum;
    }
}

/* --------------------------------------------------------- O13 leapfrog */

void orc_kick(int64_t n, double* vel, const double* acc, double dt_half) {
    for (int64_t i = 0; i < 3 * n; ++i) vel[i] += dt_half * acc[i];
}

void orc_drift(int64_t n, double* pos, const double* vel, double dt) {
    for (int64_t i = 0; i < 3 * n; ++i) pos[i] += dt * vel[i];
}

/* E = sum m v^2 / 2 + sum m phi / 2; out2 = {kinetic, potential}. */
void orc_energy(int64_t n, const double* vel, const double* mass,
                const double* pot, double* out2) {
    double ek = 0.0, ep = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double v2 = vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] +
                    vel[3 * i + 2] * vel[3 * i + 2];
        ek += 0.5 * mass[i] * v2;
        ep += 0.5 * mass[i] * pot[i];
    }
    out2[0] = ek;
    out2[1] = ep;
}

void orc_set_threads(int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int32_t orc_get_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
