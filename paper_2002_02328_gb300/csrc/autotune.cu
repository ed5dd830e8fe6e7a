// autotune.cu -- work-shape autotuner of the tile kernels (bd3mg_autotune).
//
// The tile kernels march each xy tile through a range of output slices (a
// z-chunk).  Short chunks give more CTAs to fill the 152 SMs but re-read more
// z halo; long chunks do the opposite.  The curvature pass, the one that
// dominates an iteration, has two compiled tile shapes with an FP32 gradient:
// 16 rows (one output row per thread, four CTAs per SM) and 32 rows (two rows
// per thread, less halo and per-step overhead per voxel, three CTAs per SM).
// The library's default picks the chunk from a cost model (waves of resident
// CTAs x (chunk + halo)) and 16-row tiles; the autotuner instead times every
// (chunk, tile) pair on the live GPU, for the caller's own volumes, and caches
// the winner in a JSON-lines file keyed by the problem's shape class.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/bd3mg.h"
#include "plan.h"

namespace {

// Shape class of a batch: SM count, precision and every volume's extents, PSF
// extents and slab bounds.
std::string tune_key(int nvol, const bd3mg_params *p, int sms) {
    std::ostringstream k;
    k << "v2|sms" << sms << "|prec" << p[0].precision;
    for (int v = 0; v < nvol; ++v) {
        k << "|" << p[v].nx << "x" << p[v].ny << "x" << p[v].nz << ":" << p[v].px << "x" << p[v].py << "x" << p[v].pz;
        if (p[v].nslabs > 1 && p[v].slab_bounds) {
            k << ":s";
            for (int s = 0; s <= p[v].nslabs; ++s) k << (s ? "," : "") << p[v].slab_bounds[s];
        }
    }
    return k.str();
}

// Cached (chunk, curvature rows) of `key` in the JSON-lines file; false if none.
bool cache_lookup(const char *path, const std::string &key, int *zc, int *rows) {
    std::ifstream f(path);
    if (!f) return false;
    std::string line, want = "\"key\": \"" + key + "\"";
    bool found = false;
    while (std::getline(f, line)) {
        if (line.find(want) == std::string::npos) continue;
        const size_t z = line.find("\"zchunk\": "), r = line.find("\"curv_rows\": ");
        if (z == std::string::npos || r == std::string::npos) continue;
        *zc = std::atoi(line.c_str() + z + 10);
        *rows = std::atoi(line.c_str() + r + 13);
        found = true;
    }
    return found;
}

}  // namespace

extern "C" bd3mg_status bd3mg_autotune(int nvol, const bd3mg_params *p, const float *const *y, int data_on_device,
                                       void *stream, int iters, const char *cache_path, int *zchunk,
                                       int *curv_rows, double *ms_per_iteration) {
    bd3mg::NvtxRange nvtx_("bd3mg autotune");
    if (nvol < 1 || !p || !y || !zchunk || iters < 1) return BD3MG_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return BD3MG_ECUDA;
    const std::string key = tune_key(nvol, p, sms);
    if (cache_path) {
        int z = 0, rows = 0;
        if (cache_lookup(cache_path, key, &z, &rows)) {
            *zchunk = z;
            if (curv_rows) *curv_rows = rows;
            if (ms_per_iteration) *ms_per_iteration = -1.0;
            return BD3MG_OK;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BD3MG_ECUDA;
    static const int kCandidates[] = {0, 4, 6, 8, 12, 16, 24, 32, 48};
    std::vector<int> tiles = {32};
    if (p[0].precision == BD3MG_FP32) tiles = {16, 32};
    std::vector<bd3mg_params> q(p, p + nvol);
    int best = -1, best_rows = 0;
    double best_ms = 0.0;
    std::ostringstream tried;
    bd3mg_status result = BD3MG_OK;
    for (int rows : tiles)
    for (int zc : kCandidates) {
        for (auto &qq : q) {
            qq.zchunk = zc;
            qq.curv_rows = rows;
        }
        bd3mg_ctx *c = nullptr;
        bd3mg_status st = bd3mg_batch_create(nvol, q.data(), y, nullptr, data_on_device, stream, nullptr, &c);
        if (st == BD3MG_OK) st = bd3mg_iterate_async(c, 2);                 // warm-up
        float ms = 0.f;
        if (st == BD3MG_OK) {
            cudaEventRecord(e0, s);
            st = bd3mg_iterate_async(c, iters);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                st = BD3MG_ECUDA;
        }
        bd3mg_destroy(c);
        if (st == BD3MG_ENOMEM || st == BD3MG_EINVAL) continue;              // candidate not usable here
        if (st != BD3MG_OK) {
            result = st;
            break;
        }
        const double per = ms / iters;
        tried << (tried.tellp() > 0 ? ", " : "") << "\"" << zc << "/" << rows << "\": " << per;
        if (best < 0 || per < best_ms) {
            best = zc;
            best_rows = rows;
            best_ms = per;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != BD3MG_OK) return result;
    if (best < 0) return BD3MG_EUNSUPPORTED;
    *zchunk = best;
    if (curv_rows) *curv_rows = best_rows;
    if (ms_per_iteration) *ms_per_iteration = best_ms;
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        if (f) f << "{\"key\": \"" << key << "\", \"zchunk\": " << best << ", \"curv_rows\": " << best_rows
                 << ", \"ms_per_iteration\": " << best_ms << ", \"candidates (chunk/rows)\": {" << tried.str()
                 << "}}\n";
    }
    return BD3MG_OK;
}
