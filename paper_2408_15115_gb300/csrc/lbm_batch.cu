// lbm_batch.cu -- collide+stream with a chosen tile (the autotuner's timing
// kernel) and the batched collide+stream and support-moment launches over
// the (run, block) table of many independent runs.
#include "lbm_xpair.cuh"
#include "support_moments.cuh"

namespace turret {

// Register budget variants of the collide+stream launches (two cells per
// thread), chosen by the autotuner with the tile: MINB resident 256-thread
// blocks per SM, i.e. at most 128 registers per thread for MINB = 2 (no
// spilling) and 85 for MINB = 3 (spills, more resident warps).
// K1 over one window with a chosen tile (the autotuner's timing kernel): the
// same cells and arithmetic as k_collide_stream, no window-slot carry.
template <int ST, int MODE, int MINB>
__global__ void __launch_bounds__(256, MINB) k_collide_tiled(Geom g, const typename Codec<ST>::T *__restrict__ src,
                                                       typename Codec<ST>::T *__restrict__ dst,
                                                       const float *__restrict__ utop_in,
                                                       float *__restrict__ utop_out, const DevState *st, int slot,
                                                       const float *__restrict__ hbox, BoxGeom box, int tx) {
    int cx, cy, cz;
    tile_coords(blockIdx.x, tx, g.nx, g.ny, 2, cx, cy, cz);
    k1_pair<ST, MODE>(g, src, dst, utop_in, utop_out, st->s[slot], hbox, box, cx, cy, cz);
}

// ---------------------------------------------------------------------------
// Batched K1: one launch over the (run, tile) table of many independent runs.
// Block b belongs to the run r with prefix[r] <= b < prefix[r + 1]; every run
// keeps its own storage type, window, boundary conditions, relaxation times
// and tile, read from its descriptor.  PHASE_BULK: the far cells of runs that
// split (no blocks for the others; 16-bit runs have theirs in the
// PHASE_BULK16 launch); PHASE_NEAR: the near region of runs that
// split, the whole window (with forcing) of runs that do not.
template <int PHASE, int ST>
__device__ __forceinline__ void batch_k1_run(const CollideDesc &R, int p, int lb) {
    using T = typename Codec<ST>::T;
    const Geom g = R.g;
    const BoxGeom box = R.box;
    const T *src = (const T *)R.f[p];
    T *dst = (T *)R.f[1 - p];
    const BodySlot &S = R.st->s[p];
    int cx, cy, cz;
    if (PHASE == PHASE_BULK) {
        tile_coords(lb, R.tx, g.nx, g.ny, 2, cx, cy, cz);
        k1_pair<ST, K1_FAR>(g, src, dst, R.utop[1 - p], R.utop[p], S, R.hbox, box, cx, cy, cz);
    } else if (R.split) {
        // the near region (a box of some 20-40 cells a side) as one flat range
        // of cells, x fastest: every thread has a cell but those of the last block
        const int ex = box.Bx + 2 * NEAR_GROW, ey = box.By + 2 * NEAR_GROW, ez = box.Bz + 2 * NEAR_GROW;
        const int i = lb * (int)blockDim.x + (int)threadIdx.x;
        if (i >= ex * ey * ez) return;
        cx = i % ex;
        cy = (i / ex) % ey;
        cz = i / (ex * ey);
        k1_cell<ST, K1_NEAR>(g, src, dst, R.utop[1 - p], R.utop[p], S, R.hbox, box, cx, cy, cz);
    } else {
        tile_coords(lb, R.tx, g.nx, g.ny, 2, cx, cy, cz);
        k1_pair<ST, K1_ALLF>(g, src, dst, R.utop[1 - p], R.utop[p], S, R.hbox, box, cx, cy, cz);
    }
}

// MINB: resident blocks of 256 threads per SM the register budget is sized
// for (the near phase of a large batch is thousands of blocks: 2).
template <int PHASE, int MINB>
__global__ void __launch_bounds__(256, MINB) k_batch_collide(const CollideDesc *__restrict__ runs,
                                                       const int *__restrict__ prefix, int nruns, int p) {
    // the run's descriptor is staged in shared memory (one load per thread):
    // its fields are then operands read on use rather than registers held
    // through the cell
    constexpr int NW = (int)(sizeof(CollideDesc) / 4);
    static_assert(sizeof(CollideDesc) % 4 == 0 && NW <= 128, "descriptor staged by one load per thread");
    __shared__ CollideDesc R;
    int lb;
    const int r = block_run(prefix, nruns, lb);
    if (threadIdx.x < NW)
        reinterpret_cast<int *>(&R)[threadIdx.x] = __ldg(reinterpret_cast<const int *>(runs + r) + threadIdx.x);
    __syncthreads();
    switch (R.storage) {
        case ST_F32: batch_k1_run<PHASE, ST_F32>(R, p, lb); break;
        case ST_F16: batch_k1_run<PHASE, ST_F16>(R, p, lb); break;
        default: batch_k1_run<PHASE, ST_BF16>(R, p, lb); break;
    }
}

// Batched far-cell K1 of 16-bit runs on x-adjacent pairs
// (lbm_xpair.cuh), with the register budget of the single-window x-pair
// kernel (96 registers, five 128-thread blocks per SM) rather than the FP32
// one the shared launch is held to.  A block owns a tile of tx16 x (128 /
// tx16) x 2 cells: tx16 / 2 pairs per row, then the rows, then the two planes
// over its threads; tiles the x-pair path does not admit run the one-cell
// code (thread t: column t of the tile, both planes).
template <int ST>
__device__ __forceinline__ void batch_bulk16_run(const CollideDesc &R, int p, int lb) {
    using T = typename Codec<ST>::T;
    const Geom g = R.g;  // by value: operands in registers, not re-read from the staged descriptor
    const BoxGeom box = R.box;
    const T *src = (const T *)R.f[p];
    T *dst = (T *)R.f[1 - p];
    const BodySlot &S = R.st->s[p];
    const int tw = R.tx16, th = 128 / tw, gx = (g.nx + tw - 1) / tw, gy = (g.ny + th - 1) / th;
    const int x0 = (lb % gx) * tw, y0 = ((lb / gx) % gy) * th, z0 = 2 * (lb / (gx * gy));
    const int t = (int)threadIdx.x;
    if (xpair_tile_ok<K1_FAR, true>(g, S, box, x0, y0, z0, tw, th)) {
        const int hp = tw >> 1, r = t / hp;
        xpair_cells<ST, K1_FAR>(g, src, dst, R.utop[p], S, R.hbox, box, x0 + 2 * (t % hp), y0 + r % th, z0 + r / th);
        return;
    }
    k1_cell<ST, K1_FAR>(g, src, dst, R.utop[1 - p], R.utop[p], S, R.hbox, box, x0 + t % tw, y0 + t / tw, z0);
    if (z0 + 1 < g.nz)
        k1_cell<ST, K1_FAR>(g, src, dst, R.utop[1 - p], R.utop[p], S, R.hbox, box, x0 + t % tw, y0 + t / tw, z0 + 1);
}

__global__ void __launch_bounds__(128, 5) k_batch_collide16(const CollideDesc *__restrict__ runs,
                                                            const int *__restrict__ prefix, int nruns, int p) {
    constexpr int NW = (int)(sizeof(CollideDesc) / 4);
    static_assert(sizeof(CollideDesc) % 4 == 0 && NW <= 128, "descriptor staged by one load per thread");
    __shared__ CollideDesc R;
    int lb;
    const int r = block_run(prefix, nruns, lb);
    if (threadIdx.x < NW)
        reinterpret_cast<int *>(&R)[threadIdx.x] = __ldg(reinterpret_cast<const int *>(runs + r) + threadIdx.x);
    __syncthreads();
    if (R.storage == ST_F16) batch_bulk16_run<ST_F16>(R, p, lb);
    else batch_bulk16_run<ST_BF16>(R, p, lb);
}

// Batched K2 + binning: per run nmom(r) moment blocks then its tiles, on
// f(t+1) in buffer 1 - p and window slot 1 - p (the advanced body).
__global__ void __launch_bounds__(MB_THREADS) k_batch_box_moments_bin(const RunDesc *__restrict__ runs,
                                                                      const int *__restrict__ prefix, int nruns,
                                                                      int p) {
    int lb;
    const RunDesc &R = runs[block_run(prefix, nruns, lb)];
    const Geom g = R.g;
    const BoxGeom box = R.box;
    const int nmom = (int)((box.nbox + MB_THREADS - 1) / MB_THREADS);
    const int so = 1 - p;
    switch (R.storage) {
        case ST_F32:
            mb_block<ST_F32>(g, (const float *)R.f[1 - p], R.utop[p], R.st, so, box, R.ba, nmom, R.nm, R.m.base, R.m.seg,
                             R.tile_list, R.tile_count, R.cap, R.st, R.bc.rmin, R.bc.rmax, lb);
            break;
        case ST_F16:
            mb_block<ST_F16>(g, (const __half *)R.f[1 - p], R.utop[p], R.st, so, box, R.ba, nmom, R.nm, R.m.base, R.m.seg,
                             R.tile_list, R.tile_count, R.cap, R.st, R.bc.rmin, R.bc.rmax, lb);
            break;
        default:
            mb_block<ST_BF16>(g, (const __nv_bfloat16 *)R.f[1 - p], R.utop[p], R.st, so, box, R.ba, nmom, R.nm,
                              R.m.base, R.m.seg, R.tile_list, R.tile_count, R.cap, R.st, R.bc.rmin, R.bc.rmax, lb);
            break;
    }
}

template <int ST, int MINB>
static cudaError_t tiled_t(const Geom &g, const void *src, void *dst, const float *utop_in, float *utop_out,
                           const DevState *st, int slot, const float *hbox, const BoxGeom &box, bool has_box,
                           int threads, int tx, cudaStream_t s) {
    using T = typename Codec<ST>::T;
    const int ty = threads / tx;
    const unsigned nb = (unsigned)(((g.nx + tx - 1) / tx) * ((g.ny + ty - 1) / ty) * ((g.nz + 1) / 2));
    if (has_box)
        k_collide_tiled<ST, K1_ALLF, MINB><<<nb, threads, 0, s>>>(g, (const T *)src, (T *)dst, utop_in, utop_out, st, slot, hbox, box, tx);
    else
        k_collide_tiled<ST, K1_ALL, MINB><<<nb, threads, 0, s>>>(g, (const T *)src, (T *)dst, utop_in, utop_out, st, slot, hbox, box, tx);
    return cudaGetLastError();
}

template <int MINB>
static cudaError_t tiled_m(const Geom &g, int storage, const void *src, void *dst, const float *utop_in,
                           float *utop_out, const DevState *st, int slot, const float *hbox, const BoxGeom &box,
                           bool has_box, int threads, int tx, cudaStream_t s) {
    switch (storage) {
        case ST_F32: return tiled_t<ST_F32, MINB>(g, src, dst, utop_in, utop_out, st, slot, hbox, box, has_box, threads, tx, s);
        case ST_F16: return tiled_t<ST_F16, MINB>(g, src, dst, utop_in, utop_out, st, slot, hbox, box, has_box, threads, tx, s);
        default: return tiled_t<ST_BF16, MINB>(g, src, dst, utop_in, utop_out, st, slot, hbox, box, has_box, threads, tx, s);
    }
}

bool valid_tile(int threads, int tx, int minb) {
    return (threads == 64 || threads == 128 || threads == 256) && (tx == 16 || tx == 32 || tx == 64 || tx == 128) &&
           tx <= threads && (minb == 2 || minb == 3);
}

cudaError_t launch_collide_tiled(const Geom &g, int storage, const void *src, void *dst, const float *utop_in,
                                 float *utop_out, const DevState *st, int slot, const float *hbox,
                                 const BoxGeom &box, bool has_box, int threads, int tx, int minb, cudaStream_t s) {
    if (!valid_tile(threads, tx, minb)) return cudaErrorInvalidValue;
    if (minb == 2) return tiled_m<2>(g, storage, src, dst, utop_in, utop_out, st, slot, hbox, box, has_box, threads, tx, s);
    return tiled_m<3>(g, storage, src, dst, utop_in, utop_out, st, slot, hbox, box, has_box, threads, tx, s);
}

static int tile_blocks(int ex, int ey, int ez, int threads, int tx, int pz) {
    const int ty = threads / tx;
    return ((ex + tx - 1) / tx) * ((ey + ty - 1) / ty) * ((ez + pz - 1) / pz);
}

bool bulk16_run(const RunDesc &r) {
    return r.split && (r.storage == ST_F16 || r.storage == ST_BF16) && r.g.nx % 2 == 0;
}

int bulk16_tile(const RunDesc &r) { return r.g.nx % 64 == 0 ? 64 : 32; }

int blocks_bulk(const RunDesc &r, int threads) {
    return r.split && !bulk16_run(r) ? tile_blocks(r.g.nx, r.g.ny, r.g.nz, threads, r.tx, 2) : 0;
}

int blocks_bulk16(const RunDesc &r) {
    return bulk16_run(r) ? tile_blocks(r.g.nx, r.g.ny, r.g.nz, 128, bulk16_tile(r), 2) : 0;
}

int blocks_near(const RunDesc &r, int threads) {
    if (!r.split) return tile_blocks(r.g.nx, r.g.ny, r.g.nz, threads, r.tx, 2);
    const long long cells = (long long)(r.box.Bx + 2 * NEAR_GROW) * (r.box.By + 2 * NEAR_GROW) *
                            (r.box.Bz + 2 * NEAR_GROW);
    return (int)((cells + threads - 1) / threads);
}

int blocks_box_moments_bin(const RunDesc &r) {
    return (int)((r.box.nbox + MB_THREADS - 1) / MB_THREADS) + r.box.tx * r.box.ty * r.box.tz;
}

cudaError_t launch_batch_collide(int phase, const CollideDesc *runs, const int *prefix, int nruns, int p,
                                 int nblocks, int threads, int minb, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    if (phase == PHASE_BULK16)
        k_batch_collide16<<<nblocks, 128, 0, s>>>(runs, prefix, nruns, p);
    else if (phase == PHASE_NEAR)
        k_batch_collide<PHASE_NEAR, 2><<<nblocks, threads, 0, s>>>(runs, prefix, nruns, p);
    else if (minb == 2)
        k_batch_collide<PHASE_BULK, 2><<<nblocks, threads, 0, s>>>(runs, prefix, nruns, p);
    else
        k_batch_collide<PHASE_BULK, 3><<<nblocks, threads, 0, s>>>(runs, prefix, nruns, p);
    return cudaGetLastError();
}

bool is_batch_bulk_kernel(const void *fn) {
    return fn == (const void *)k_batch_collide<PHASE_BULK, 2> || fn == (const void *)k_batch_collide<PHASE_BULK, 3> ||
           fn == (const void *)k_batch_collide16;
}

cudaError_t launch_batch_box_moments_bin(const RunDesc *runs, const int *prefix, int nruns, int p, int nblocks,
                                         cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    k_batch_box_moments_bin<<<nblocks, MB_THREADS, 0, s>>>(runs, prefix, nruns, p);
    return cudaGetLastError();
}

}  // namespace turret
