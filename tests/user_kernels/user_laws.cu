// User interaction laws compiled against fdps_user_force.cuh (test code):
// softened gravity with monopole or quadrupole superparticles written as a
// user would write it, and a law that only counts the list entries.
#include "fdps_user_force.cuh"

using fdps_user::Epi;
using fdps_user::Epj;
using fdps_user::Spj;

namespace {

struct GravForce {
    float ax, ay, az, pot;
    __device__ void clear() { ax = ay = az = pot = 0.f; }
};

// a_i += m (x_j - x_i) / (r^2 + eps_i^2)^{3/2}, phi_i -= m / (r^2 + eps_i^2)^{1/2};
// superparticles with their traceless quadrupole (r = x_i - com, R^2 = r^2 + eps_i^2):
// phi -= M/R + r.Q.r / (2 R^5), a += -M r/R^3 + Q r/R^5 - 5/2 (r.Q.r) r/R^7
struct Gravity {
    __device__ void operator()(const Epi& i, const Epj* j, int nj, GravForce& f) const {
        for (int k = 0; k < nj; ++k) {
            const float dx = j[k].x - i.x, dy = j[k].y - i.y, dz = j[k].z - i.z;
            const float r2 = dx * dx + dy * dy + dz * dz + i.eps2;
            const float ri = rsqrtf(r2);
            const float mri = j[k].m * ri;
            const float mri3 = mri * ri * ri;
            f.ax += mri3 * dx;
            f.ay += mri3 * dy;
            f.az += mri3 * dz;
            f.pot -= mri;
        }
    }
    __device__ void operator()(const Epi& i, const Spj* j, int nj, GravForce& f) const {
        for (int k = 0; k < nj; ++k) {
            const Spj& s = j[k];
            const float rx = i.x - s.x, ry = i.y - s.y, rz = i.z - s.z;
            const float R2 = rx * rx + ry * ry + rz * rz + i.eps2;
            const float Ri = rsqrtf(R2);
            const float Ri2 = Ri * Ri, Ri3 = Ri * Ri2, Ri5 = Ri3 * Ri2;
            const float qx = s.qxx * rx + s.qxy * ry + s.qxz * rz;
            const float qy = s.qxy * rx + s.qyy * ry + s.qyz * rz;
            const float qz = s.qxz * rx + s.qyz * ry + s.qzz * rz;
            const float rqr = rx * qx + ry * qy + rz * qz;
            const float c = s.m * Ri3 + 2.5f * rqr * Ri5 * Ri2;
            f.ax += qx * Ri5 - c * rx;
            f.ay += qy * Ri5 - c * ry;
            f.az += qz * Ri5 - c * rz;
            f.pot -= s.m * Ri + 0.5f * rqr * Ri5;
        }
    }
};

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
    const cudaError_t e = fdps_user::calc_force(v, Gravity{}, Gravity{}, static_cast<GravForce*>(out),
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
