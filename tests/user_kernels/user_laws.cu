// User interaction laws compiled against fdps_user_force.cuh (test code):
// softened gravity with monopole or quadrupole superparticles written as a
// user would write it, and a law that only counts the list entries.
#include "fdps_user_force.cuh"

using fdps_user::Epi;
using fdps_user::Epj;
using fdps_user::Spj;

#include "gravity_law.inc"  // struct Force, struct Law: softened gravity

namespace {

struct CountForce {
    unsigned int n_epj, n_spj;
    __device__ void clear() { n_epj = n_spj = 0u; }
};

struct Count {
    __device__ void operator()(const Epi&, const Epj*, int nj, CountForce& f) const { f.n_epj += nj; }
    __device__ void operator()(const Epi&, const Spj*, int nj, CountForce& f) const { f.n_spj += nj; }
};

}  // namespace

extern "C" {

// out: device float4 [n] (ax, ay, az, phi) in the caller's rows
int user_gravity(const fdps_tree* tree, const fdps_psys* ps, void* out, void* stream) {
    fdps_tree_view v;
    const int rc = fdps_tree_get_view(tree, ps, &v);
    if (rc != FDPS_OK) return rc;
    const cudaError_t e = fdps_user::calc_force(v, Law{}, Law{}, static_cast<Force*>(out),
                                                static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FDPS_OK : FDPS_ECUDA;
}

// out: device uint2 [n] (particles of opened leaves, superparticles) per row
int user_count(const fdps_tree* tree, const fdps_psys* ps, void* out, void* stream) {
    fdps_tree_view v;
    const int rc = fdps_tree_get_view(tree, ps, &v);
    if (rc != FDPS_OK) return rc;
    const cudaError_t e = fdps_user::calc_force(v, Count{}, Count{}, static_cast<CountForce*>(out),
                                                static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FDPS_OK : FDPS_ECUDA;
}

}  // extern "C"
