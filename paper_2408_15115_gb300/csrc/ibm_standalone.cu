// ibm_standalone.cu -- the spreading operator of the immersed-boundary method
// (Sec. 2.2, step l = 1) as a standalone call on a caller grid:
//   field(x) = S[h](x) = sum_k h_k W(x - X_k) dS_k.
// It runs the same gather kernel as the time step (k_spread, one block per
// 4^3 tile, candidate lists in marker order: reproducible, no atomics) with
// the grid itself as the support box.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/turret.h"
#include "turret_internal.cuh"

using namespace turret;

namespace {

__device__ __forceinline__ float pk_in(float a) { return 0.125f * (3.0f - 2.0f * a + sqrtf(1.0f + 4.0f * a - 4.0f * a * a)); }
__device__ __forceinline__ float pk_out(float a) {
    return 0.125f * (5.0f - 2.0f * a - sqrtf(fmaxf(0.0f, -7.0f + 12.0f * a - 4.0f * a * a)));
}

// Stencil record of every marker from its position: base = floor(X) - 1 and
// the four 1-D Peskin weights per axis; h dS for the gather.  A stencil that
// leaves the grid (or a non-finite position) is parked at the origin with zero
// weights and flags *err.
__global__ void k_records(int nm, const float *__restrict__ X, const float *__restrict__ h,
                          const float *__restrict__ dS, BoxGeom box, MRec *rec, int *mbase, int *err) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nm) return;
    const int B[3] = {box.Bx, box.By, box.Bz};
    MRec r;
    int bv[3];
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = X[a * nm + k];
        const float fl = floorf(x);
        const float t = x - fl;
        int b = (int)fl - 1;
        float w4[4] = {pk_out(1.0f + t), pk_in(t), pk_in(1.0f - t), pk_out(2.0f - t)};
        if (!isfinite(x) || b < 0 || b > B[a] - 4) {
            b = 0;
            w4[0] = w4[1] = w4[2] = w4[3] = 0.0f;
            bad = true;
        }
        bv[a] = b;
        float *dst = (a == 0) ? r.wx : (a == 1) ? r.wy : r.wz;
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = w4[q];
    }
    r.base = bv[0] | (bv[1] << 10) | (bv[2] << 20);
    const float d = bad ? 0.0f : dS[k];
    r.hdS[0] = h[k] * d;
    r.hdS[1] = h[nm + k] * d;
    r.hdS[2] = h[2 * nm + k] * d;
    rec[k] = r;
    mbase[k] = r.base;
    if (bad) atomicExch(err, 1);
}

// For one 4^3 tile, the markers whose stencil overlaps it, in marker order.
__global__ void __launch_bounds__(256) k_tile_lists(BoxGeom box, int nm, const int *__restrict__ mbase,
                                                    int *__restrict__ tile_list, int *__restrict__ tile_count,
                                                    int cap, int *err) {
    const int tile = blockIdx.x;
    const int tx = tile % box.tx, ty = (tile / box.tx) % box.ty, tz = tile / (box.tx * box.ty);
    const int t0[3] = {TILE * tx, TILE * ty, TILE * tz};
    __shared__ int wcount[8];
    __shared__ int total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) total = 0;
    __syncthreads();
    for (int chunk = 0; chunk < nm; chunk += 256) {
        const int k = chunk + tid;
        bool hit = false;
        if (k < nm) {
            const int pb = __ldg(mbase + k);
            const int b[3] = {pb & 1023, (pb >> 10) & 1023, (pb >> 20) & 1023};
            hit = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) hit = hit && (b[a] + 3 >= t0[a]) && (b[a] <= t0[a] + TILE - 1);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) wcount[warp] = __popc(bal);
        __syncthreads();
        int off = total;
        for (int w = 0; w < warp; ++w) off += wcount[w];
        if (hit) {
            const int pos = off + __popc(bal & ((1u << lane) - 1u));
            if (pos < cap) tile_list[(size_t)tile * cap + pos] = k;
        }
        __syncthreads();
        if (tid == 0) {
            int s = 0;
            for (int w = 0; w < 8; ++w) s += wcount[w];
            total += s;
        }
        __syncthreads();
    }
    if (tid == 0) {
        tile_count[tile] = total < cap ? total : cap;
        if (total > cap) atomicExch(err, 2);
    }
}

struct SpreadLayout {
    BoxGeom box;
    int cap;
    size_t ntiles;
    size_t off_rec, off_base, off_list, off_count, off_err, bytes;
};

bool spread_layout(int32_t nx, int32_t ny, int32_t nz, int64_t nm, SpreadLayout &L) {
    if (nx < 4 || ny < 4 || nz < 4 || nx > 1023 || ny > 1023 || nz > 1023 || nm <= 0 || nm >= (1 << 24)) return false;
    L.box.Bx = nx;
    L.box.By = ny;
    L.box.Bz = nz;
    L.box.tx = (nx + TILE - 1) / TILE;
    L.box.ty = (ny + TILE - 1) / TILE;
    L.box.tz = (nz + TILE - 1) / TILE;
    L.box.nbox = (long long)nx * ny * nz;
    L.cap = (int)(nm < MAX_CANDIDATES ? nm : MAX_CANDIDATES);
    L.ntiles = (size_t)L.box.tx * L.box.ty * L.box.tz;
    size_t off = 0;
    auto take = [&](size_t b) {
        off = (off + 255) & ~(size_t)255;
        const size_t o = off;
        off += b;
        return o;
    };
    L.off_rec = take((size_t)nm * sizeof(MRec));
    L.off_base = take((size_t)nm * 4);
    L.off_list = take(L.ntiles * (size_t)L.cap * 4);
    L.off_count = take(L.ntiles * 4);
    L.off_err = take(4);
    L.bytes = off;
    return true;
}

}  // namespace

// Enqueues the three kernels on the given scratch, waits for the stream and
// reads back the error word.
static turret_status run_spread(const float *X, const float *h, const float *dS, int64_t nm, int32_t nx, int32_t ny,
                                int32_t nz, float *field, char *scratch, const SpreadLayout &L, cudaStream_t s) {
    MRec *rec = (MRec *)(scratch + L.off_rec);
    int *mbase = (int *)(scratch + L.off_base);
    int *list = (int *)(scratch + L.off_list);
    int *count = (int *)(scratch + L.off_count);
    int *err = (int *)(scratch + L.off_err);
    if (cudaMemsetAsync(err, 0, 4, s) != cudaSuccess) return TURRET_ECUDA;
    k_records<<<(unsigned)((nm + 127) / 128), 128, 0, s>>>((int)nm, X, h, dS, L.box, rec, mbase, err);
    k_tile_lists<<<(unsigned)L.ntiles, 256, 0, s>>>(L.box, (int)nm, mbase, list, count, L.cap, err);
    MarkerArrays m;
    memset(&m, 0, sizeof m);
    m.rec = rec;
    BoxArrays ba;
    ba.u = ba.s = ba.p = nullptr;
    ba.h = field;
    if (launch_spread(L.box, (int)nm, m, ba, list, count, L.cap, s) != cudaSuccess) return TURRET_ECUDA;
    int herr = 0;
    if (cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return TURRET_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TURRET_ECUDA;
    if (herr == 1) return TURRET_EDOMAIN;
    if (herr == 2) return TURRET_EOVERFLOW;
    return TURRET_OK;
}

extern "C" size_t ibm_spread_workspace_bytes(int32_t nx, int32_t ny, int32_t nz, int64_t n_markers) {
    SpreadLayout L;
    if (!spread_layout(nx, ny, nz, n_markers, L)) return 0;
    return L.bytes + 256;
}

extern "C" turret_status ibm_spread(const float *X, const float *h, const float *dS, int64_t n_markers, int32_t nx,
                                    int32_t ny, int32_t nz, float *field, void *workspace, size_t workspace_bytes,
                                    void *stream) {
    SpreadLayout L;
    if (!X || !h || !dS || !field || !spread_layout(nx, ny, nz, n_markers, L)) return TURRET_EINVAL;
    if (!workspace || workspace_bytes < L.bytes) return TURRET_ENOMEM;
    if (((uintptr_t)workspace & 255) != 0) return TURRET_EINVAL;
    return run_spread(X, h, dS, n_markers, nx, ny, nz, field, (char *)workspace, L, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// ibm_spread for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc at all: code that runs
// under a host framework whose memory pool owns the whole device, plugins that
// get no allocator from their host, and real-time loops that forbid
// allocation (and its implicit synchronisation) after start-up.  For them this
// entry point takes its scratch from a fixed array in the library's device
// image instead of a caller workspace.  The array is NOALLOC_SCRATCH_BYTES
// (8 MiB) and is held by every GPU that loads the library until the process
// exits.  The address of the array is a device address only on the device:
// host code obtains it once per device with cudaGetSymbolAddress (on the
// first call made with that device current) and passes it to the kernels.
// The cached address is valid for as long as the device's primary context
// lives: cudaDeviceReset unloads the image, and the entry point must not be
// called on that device afterwards.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[NOALLOC_MAX_DEVICES];

extern "C" turret_status ibm_spread_noalloc(const float *X, const float *h, const float *dS, int64_t n_markers,
                                            int32_t nx, int32_t ny, int32_t nz, float *field, void *stream) {
    SpreadLayout L;
    if (!X || !h || !dS || !field || !spread_layout(nx, ny, nz, n_markers, L)) return TURRET_EINVAL;
    if (L.bytes > NOALLOC_SCRATCH_BYTES) return TURRET_ENOMEM;  // beyond the fixed scratch
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return TURRET_ECUDA;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TURRET_ECUDA;
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    // run_spread clears the error word first; records, lists and counts are
    // fully rewritten by every call
    return run_spread(X, h, dS, n_markers, nx, ny, nz, field, (char *)scratch, L, (cudaStream_t)stream);
}
