/*
 * fdps_oracle.h -- TEST INFRASTRUCTURE ONLY: the FP64 CPU oracle of the
 * Barnes-Hut tree force (FDPS, Iwasawa et al. 2016).  See fdps_oracle.c for
 * the definitions each function follows.  Positions, accelerations and
 * centres of mass are row-major [n][3] doubles; quadrupoles are [n][6] in
 * the order xx, yy, zz, xy, xz, yz.
 */
#ifndef FDPS_ORACLE_H
#define FDPS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_tree orc_tree;

int orc_root_box(int64_t n, const double* pos, double* lo3, double* L, double* s);
uint64_t orc_morton(uint32_t qx, uint32_t qy, uint32_t qz);
void orc_keys(int64_t n, const double* pos, const double* lo3, double s,
              uint64_t* keys, uint32_t* q3);
void orc_sort(int64_t n, const uint64_t* keys, uint32_t* perm);
void orc_quadrupole(int64_t n, const double* pos, const double* mass,
                    const double* c, double* Q);
void orc_multipole(int64_t n, const double* pos, const double* mass,
                   double* M, double* com, double* Q);
void orc_spj_force(const double* xi, double ep2, double M, const double* com,
                   const double* Q, double* acc3, double* pot);

orc_tree* orc_tree_build(int64_t n, const double* pos, const double* mass,
                         const double* eps, double theta, int32_t n_leaf,
                         int32_t n_grp, int32_t quad);
void orc_tree_free(orc_tree* t);
int64_t orc_tree_n_nodes(const orc_tree* t);
int64_t orc_tree_n_groups(const orc_tree* t);
void orc_tree_box(const orc_tree* t, double* out5);
void orc_tree_keys(const orc_tree* t, uint64_t* keys_in, uint32_t* perm);
void orc_tree_nodes(const orc_tree* t, int32_t* level, uint64_t* prefix,
                    int64_t* first, int64_t* count, int64_t* child_first,
                    int32_t* nchild, double* mass, double* com, double* quad);
void orc_tree_groups(const orc_tree* t, int64_t* first, int64_t* count,
                     int64_t* node, double* box6, uint32_t* qbox6);
int orc_open_cell(const orc_tree* t, int64_t node, int64_t group);
int64_t orc_tree_walk(const orc_tree* t, int64_t group, int64_t* epj,
                      int64_t cap_epj, int64_t* n_epj, int64_t* spj,
                      int64_t cap_spj, int64_t* n_spj);
void orc_tree_force(const orc_tree* t, const int64_t* gidx, int64_t ng,
                    double* acc_in, double* pot_in, int64_t* totals);

void orc_direct(int64_t n, const double* pos, const double* mass,
                const double* eps, const int64_t* idx, int64_t ni,
                double* acc, double* pot);
/* short-range mode: Wendland C6 kernel (3D, support radius H) and the
   brute-force neighbour counts and SPH density of rows idx (all if NULL);
   mode 0 fixed r_fixed, 1 h_i, 2 h_j, 3 max(h_i, h_j) */
double orc_wendland_c6(double r, double H);
void orc_wendland_c6_array(int64_t n, const double* r, double H, double* out);
void orc_neighbors(int64_t n, const double* pos, const double* mass, const double* h,
                   int32_t mode, double r_fixed, const int64_t* idx, int64_t ni,
                   int64_t* count, double* rho);
void orc_kick(int64_t n, double* vel, const double* acc, double dt_half);
void orc_drift(int64_t n, double* pos, const double* vel, double dt);
void orc_energy(int64_t n, const double* vel, const double* mass,
                const double* pot, double* out2);
void orc_set_threads(int32_t nthreads);
int32_t orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
