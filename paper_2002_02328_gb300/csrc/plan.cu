// plan.cu -- host-side planning helpers (PSF factoring, slab colouring,
// z-chunk choice, TMA descriptor encoding).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "kernels.cuh"
#include "plan.h"

namespace bd3mg {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3D tile map over a pitched float32 volume: dims (nx, ny, nz), box (bx, by, 1),
// zero fill outside the volume.
}  // namespace

bool encode_map(CUtensorMap *m, const void *base, int esize, int nx, int ny, int nz, int pitch, int bx, int by) {
    auto fn = encode_fn();
    if (!fn || (esize != 4 && esize != 2)) return false;
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)pitch * esize, (cuuint64_t)pitch * esize * (cuuint64_t)ny};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                    const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}


// 5-D tile map over channels-last BF16 activations [B][D][H][W][ld] reading
// channels [0, C) of each row: box 8 channels x bx x by x bz x 1, zero fill
// outside the volume (the zero padding of a 3x3x3 convolution).
bool encode_act_map(CUtensorMap *m, const void *base, int C, int ld, int W, int H, int D, int B, int bx, int by,
                    int bz) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t row = (cuuint64_t)ld * 2;
    cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)B};
    cuuint64_t strides[4] = {row, row * W, row * W * H, row * W * H * D};
    cuuint32_t box[5] = {8, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Rank-1 factoring of each depth's PSF in FP64: with m_x(a) = sum_{b,c} h,
// m_y, m_z the marginals and S = sum h, a rank-1 tensor satisfies
// h = m_x m_y m_z / S^2.  Factors: fx = m_x / S, fy = m_y / S, fz = m_z,
// written zero-padded to radii (R, RZ) into fx [nz][2R+1], fy [nz][2R+1],
// fz [nz][2RZ+1].  Uses no heap memory.
bool factor_psf_into(const bd3mg_params &p, int R, int RZ, float *fx, float *fy, float *fz, double *worst) {
    const int rx = (p.px - 1) / 2, ry = (p.py - 1) / 2, rz = (p.pz - 1) / 2;
    const int kxy = 2 * R + 1, kz = 2 * RZ + 1;
    if (p.px > kMaxPsfExtent || p.py > kMaxPsfExtent || p.pz > kMaxPsfExtent || rx > R || ry > R || rz > RZ)
        return false;
    std::fill(fx, fx + (size_t)p.nz * kxy, 0.f);
    std::fill(fy, fy + (size_t)p.nz * kxy, 0.f);
    std::fill(fz, fz + (size_t)p.nz * kz, 0.f);
    *worst = 0.0;
    double mx[kMaxPsfExtent], my[kMaxPsfExtent], mz[kMaxPsfExtent];
    for (int z = 0; z < p.nz; ++z) {
        const float *h = p.psf + (size_t)z * p.pz * p.py * p.px;
        std::fill(mx, mx + p.px, 0.0);
        std::fill(my, my + p.py, 0.0);
        std::fill(mz, mz + p.pz, 0.0);
        double S = 0.0, hmax = 0.0;
        for (int c = 0; c < p.pz; ++c)
            for (int b = 0; b < p.py; ++b)
                for (int a = 0; a < p.px; ++a) {
                    const double v = h[((size_t)c * p.py + b) * p.px + a];
                    mx[a] += v;
                    my[b] += v;
                    mz[c] += v;
                    S += v;
                    hmax = std::max(hmax, std::fabs(v));
                }
        if (hmax == 0.0) continue;              // all-zero PSF: zero factors
        if (S == 0.0) return false;
        double res = 0.0;
        for (int c = 0; c < p.pz; ++c)
            for (int b = 0; b < p.py; ++b)
                for (int a = 0; a < p.px; ++a) {
                    const double v = h[((size_t)c * p.py + b) * p.px + a];
                    res = std::max(res, std::fabs(v - mx[a] * my[b] * mz[c] / (S * S)));
                }
        *worst = std::max(*worst, res / hmax);
        if (res > 1e-6 * hmax) return false;
        for (int a = 0; a < p.px; ++a) fx[(size_t)z * kxy + (a - rx) + R] = (float)(mx[a] / S);
        for (int b = 0; b < p.py; ++b) fy[(size_t)z * kxy + (b - ry) + R] = (float)(my[b] / S);
        for (int c = 0; c < p.pz; ++c) fz[(size_t)z * kz + (c - rz) + RZ] = (float)mz[c];
    }
    return true;
}

bool factor_psf(const bd3mg_params &p, int R, int RZ, std::vector<float> &fx, std::vector<float> &fy,
                std::vector<float> &fz, double *worst) {
    fx.assign((size_t)p.nz * (2 * R + 1), 0.f);
    fy.assign((size_t)p.nz * (2 * R + 1), 0.f);
    fz.assign((size_t)p.nz * (2 * RZ + 1), 0.f);
    return factor_psf_into(p, R, RZ, fx.data(), fy.data(), fz.data(), worst);
}

// Bound on the Lipschitz constant of grad f from the factored PSF of one volume
// (factor rows of length 2R+1, 2RZ+1 per output depth): ||H||_2^2 <= ||H||_1 ||H||_inf,
// the largest absolute column sum (every output depth z = zi + c reading input
// depth zi) times the largest absolute row sum; plus 2 eta and the penalty's
// Hessian bound lambda / delta times sum_a ||V^a||^2 <= 12 (8 for the joint X-Y
// term of mode 1, which adds 2 kappa ||V^Z||^2 <= 8 kappa).
double lipschitz_bound(const bd3mg_params &p, int R, int RZ, const std::vector<float> &fx,
                       const std::vector<float> &fy, const std::vector<float> &fz) {
    const int kxy = 2 * R + 1, kz = 2 * RZ + 1;
    auto absum = [](const float *v, int n) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += std::fabs((double)v[i]);
        return s;
    };
    std::vector<double> sxy(p.nz);
    double rowmax = 0.0;
    for (int z = 0; z < p.nz; ++z) {
        sxy[z] = absum(&fx[(size_t)z * kxy], kxy) * absum(&fy[(size_t)z * kxy], kxy);
        rowmax = std::max(rowmax, sxy[z] * absum(&fz[(size_t)z * kz], kz));
    }
    double colmax = 0.0;
    for (int zi = 0; zi < p.nz; ++zi) {
        double s = 0.0;
        for (int c = -RZ; c <= RZ; ++c) {
            const int z = zi + c;
            if (z < 0 || z >= p.nz) continue;
            s += sxy[z] * std::fabs((double)fz[(size_t)z * kz + c + RZ]);
        }
        colmax = std::max(colmax, s);
    }
    const double pen = p.penalty == BD3MG_PENALTY_JOINT_XY ? 8.0 * p.lambda / p.delta + 8.0 * p.kappa
                                                            : 12.0 * p.lambda / p.delta;
    return rowmax * colmax + 2.0 * p.eta + pen;
}

// The same bound from the dense PSF (host taps [nz][pz][py][px]): the row sum of
// output depth z is sum |h_z|, the column sum of input depth zi sums the taps
// h_{zi+c}(., ., c) of every output depth that reads it.
double lipschitz_bound_dense(const bd3mg_params &p) {
    const size_t per = (size_t)p.px * p.py;
    const int rz = (p.pz - 1) / 2;
    double rowmax = 0.0, colmax = 0.0;
    std::vector<double> plane_sum((size_t)p.nz * p.pz, 0.0);     // [z][c]: sum over a, b of |h_z(a, b, c)|
    for (int z = 0; z < p.nz; ++z) {
        double row = 0.0;
        for (int c = 0; c < p.pz; ++c) {
            double t = 0.0;
            const float *h = p.psf + ((size_t)z * p.pz + c) * per;
            for (size_t k = 0; k < per; ++k) t += std::fabs((double)h[k]);
            plane_sum[(size_t)z * p.pz + c] = t;
            row += t;
        }
        rowmax = std::max(rowmax, row);
    }
    for (int zi = 0; zi < p.nz; ++zi) {
        double col = 0.0;
        for (int c = -rz; c <= rz; ++c) {
            const int z = zi + c;
            if (z >= 0 && z < p.nz) col += plane_sum[(size_t)z * p.pz + c + rz];
        }
        colmax = std::max(colmax, col);
    }
    const double pen = p.penalty == BD3MG_PENALTY_JOINT_XY ? 8.0 * p.lambda / p.delta + 8.0 * p.kappa
                                                            : 12.0 * p.lambda / p.delta;
    return rowmax * colmax + 2.0 * p.eta + pen;
}

// Greedy colouring in increasing z: a slab takes the first colour whose slabs
// all end at least `gap` slices before it starts.  Slabs of one colour then
// read and write disjoint data, so updating them together equals updating them
// one after the other.
int colour_slabs(const std::vector<int> &bounds, int gap, std::vector<int> &colour) {
    const int ns = (int)bounds.size() - 1;
    colour.assign(ns, 0);
    std::vector<int> last_end;                  // per colour: end slice of its last slab
    for (int s = 0; s < ns; ++s) {
        int c = 0;
        for (; c < (int)last_end.size(); ++c)
            if (bounds[s] - last_end[c] >= gap) break;
        if (c == (int)last_end.size()) last_end.push_back(0);
        colour[s] = c;
        last_end[c] = bounds[s + 1];
    }
    return (int)last_end.size();
}


int choose_zchunk(long long slots, int ntiles, int halo, const std::vector<std::pair<int, int>> &ranges) {
    return choose_zchunk(slots, ntiles, halo, ranges.data(), (int)ranges.size());
}

int choose_zchunk(long long slots, int ntiles, int halo, const std::pair<int, int> *ranges, int nranges) {
    slots = std::max<long long>(1, slots);
    long long best_cost = -1;
    int best = 4;
    for (int zc = 4; zc <= ZC_MAX; ++zc) {
        long long items = 0;
        int longest = 0;
        for (int i = 0; i < nranges; ++i) {
            const auto &r = ranges[i];
            const int len = r.second - r.first;
            if (len <= 0) continue;
            const int nch = (len + zc - 1) / zc;
            items += (long long)nch * ntiles;
            longest = std::max(longest, (len + nch - 1) / nch);
        }
        const long long cost = ((items + slots - 1) / slots) * (longest + halo);
        if (best_cost < 0 || cost <= best_cost) {
            best_cost = cost;
            best = zc;
        }
    }
    return best;
}

}  // namespace bd3mg
