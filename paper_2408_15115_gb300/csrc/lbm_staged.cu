// lbm_staged.cu -- the bulk collide+stream with 16-bit population storage,
// its sources and results moved through shared memory by the tensor memory
// accelerator (opt-in: flags.staged_loads).
//
// With FP16 / BF16 storage, cell pairs (z, z + 1) move every population with
// 2-byte accesses, which on this part stream at about 5 TB/s where 4- and
// 16-byte accesses reach the copy bandwidth (the default kernel therefore
// pairs x-adjacent cells and moves 4-byte words, lbm_xpair.cuh).  Here the
// data moves in bulk tensor copies instead.  A block of four computing warps
// and one producer warp works through a column of STG_TPB tiles of 32 x 4 x 2
// cells (two planes, one cell pair per thread), stacked in z.
// Population i of a tile pulls from the tile shifted by -xi_i: the producer
// issues the source boxes as 4-D bulk tensor copies (x, y, z, population)
// into an input stage, each box widened to 48 x 4 x 2 so that it starts on a
// 16-byte boundary at x0 - 8 and covers the +-1 x-shifts, the three
// populations that differ only in xi_x in one copy (nine per tile).  The
// computing warps read their 54 values at fixed shared-memory offsets, run the
// same collision as every other path (k1_pair_collide_store), write the 16-bit
// results to an output tile, and the producer stores it with one bulk tensor
// copy.  Stages and output tiles are handed over with mbarriers (full / empty
// per stage, full / empty per output tile).  Results are bitwise identical to
// the default kernel.
//
// Measured on the 256 x 256 x 512 window, FP16: cell pairs with 2-byte
// accesses 0.91 ms per launch, this pipeline 1.6 ms (1.2 ms in a variant
// without warp specialisation), the default x-pair kernel 0.71 ms: at 16-bit
// storage the collision's FP32 arithmetic sets a floor of its own, and the
// shared memory that the staged tiles in flight need leaves too few computing
// warps per SM to reach it.
//
// Periodic x / y edges: the copies read zeros outside the window; the few
// elements a tile at a periodic edge needs from the far side (one column per
// shifted population for x, one row per shifted population for y) are then
// fetched with plain loads.  Tiles that touch a closed face, the bottom or top
// boundary planes, the plane entering the ring window, the physical wrap of
// the ring, or (far-cell launches) the near region run the plain pull and
// stores.  Every wait is bounded: past the limit the kernel latches a timeout
// in the device status, waits (bounded) for its copies in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "lbm_cell.cuh"

namespace turret {

namespace {

constexpr int STG_TX = 32, STG_TY = 4, STG_TZ = 2;
constexpr int STG_TPB = 16;                        // tiles per block, stacked in z
constexpr int STG_NS = 2;                          // input stages
constexpr int STG_NO = 2;                          // output tiles
constexpr int STG_CONS = STG_TX * STG_TY;          // consumer threads (4 warps); one producer warp
constexpr int STG_BX = STG_TX + 16;               // source box width: x0 - 8 .. x0 + 40
constexpr int STG_BOX = STG_BX * STG_TY * STG_TZ;  // elements per source box
constexpr int STG_OBOX = STG_TX * STG_TY * STG_TZ; // elements per output box
constexpr unsigned STG_BYTES = 27u * STG_BOX * 2u;  // transaction bytes of one tile's sources
// dynamic shared memory: input stages, output tiles, and the mbarriers full /
// empty per stage and full / empty per output tile
constexpr size_t STG_SMEM = (STG_NS * 27 * STG_BOX + STG_NO * 27 * STG_OBOX) * 2 + (2 * STG_NS + 2 * STG_NO) * 8;
// Bounded wait on the copies (try_wait polls, each of which may suspend the
// thread for a while): ample for a few microseconds of traffic.
constexpr unsigned STG_WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// barrier 1 over the consumer warps only
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(STG_CONS) : "memory"); }

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// One 4-D tiled bulk copy global -> shared, completing on the mbarrier.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// One 4-D tiled bulk copy shared -> global (bulk async-group completion).
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, const void *src, int c0, int c1, int c2, int c3) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                     reinterpret_cast<unsigned long long>(map)),
                 "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the source shared memory of every committed store may be reused
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed store has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// shared-memory writes of this thread made visible to the bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int ST>
__device__ __forceinline__ float from_bits(unsigned short b);
template <>
__device__ __forceinline__ float from_bits<ST_F16>(unsigned short b) {
    return __half2float(__ushort_as_half(b));
}
template <>
__device__ __forceinline__ float from_bits<ST_BF16>(unsigned short b) {
    return __bfloat162float(__ushort_as_bfloat16(b));
}

// 16-bit storage encoding of a post-collision value (Codec<ST>::store), or
// with BF16 stochastic rounding the 16 random bits rnd added below the kept
// bits (store_bf16_sr).
template <int ST>
__device__ __forceinline__ unsigned short to_bits(float r);
template <>
__device__ __forceinline__ unsigned short to_bits<ST_F16>(float r) {
    return __half_as_ushort(__float2half_rn(r));
}
template <>
__device__ __forceinline__ unsigned short to_bits<ST_BF16>(float r) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(r));
}

__device__ __forceinline__ int wrap(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// Whether the cells [c0, c0 + len) of one axis meet the near region (its
// relative coordinates 0 .. ext - 1 from the support box origin lo / lo_w
// less NEAR_GROW), as the per-cell test of k1_pair does cell by cell.
__device__ __forceinline__ bool meets_near(int c0, int len, int lo, int lo_w, int ext, int n, bool periodic) {
    const int r0 = rel_axis(c0, lo, lo_w, NEAR_GROW, n, periodic);
    return periodic ? (r0 < ext || r0 + len > n) : (r0 < ext && r0 + len > 0);
}

// Whether the tile (x0, y0, z0) of the 32 x 4 x 2 tiling is staged, and the
// physical plane zp[ez] of the first row of the source boxes with xi_z =
// ez - 1 (block-uniform: every thread computes the same).
template <int MODE>
__device__ __forceinline__ bool tile_staged(const Geom &g, const BodySlot &S, const BoxGeom &box, int x0, int y0,
                                            int z0, int zp[3]) {
    bool ok = z0 >= 1 && z0 + STG_TZ + 1 <= g.nz;  // sources on interior planes z0 - 1 .. z0 + 2
#pragma unroll
    for (int ez = 0; ez < 3; ++ez) {
        zp[ez] = zphys(z0 - (ez - 1), S.ring, g.nz);
        ok = ok && zp[ez] != g.nz - 1 && zp[ez] != S.reseed && zp[ez] + 1 != S.reseed;
    }
    if (g.bc_x != BC_PERIODIC && (x0 == 0 || x0 + STG_TX == g.nx)) ok = false;
    if (g.bc_y != BC_PERIODIC && (y0 == 0 || y0 + STG_TY == g.ny)) ok = false;
    if (MODE == K1_FAR && ok) {
        const bool near =
            meets_near(x0, STG_TX, S.box_lo[0], S.box_lo_w[0], box.Bx + 2 * NEAR_GROW, g.nx, g.bc_x == BC_PERIODIC) &&
            meets_near(y0, STG_TY, S.box_lo[1], S.box_lo_w[1], box.By + 2 * NEAR_GROW, g.ny, g.bc_y == BC_PERIODIC) &&
            meets_near(z0, STG_TZ, S.box_lo[2], S.box_lo_w[2], box.Bz + 2 * NEAR_GROW, g.nz,
                       g.bc_bottom == BC_PERIODIC);
        ok = !near;
    }
    return ok;
}

}  // namespace

// Issue the 27 source boxes of the tile (x0, y0, zp) into one input stage
// (one thread).
// The three populations with the same (xi_y, xi_z) (consecutive indices
// i = ex + 3 ey + 9 ez) share their source box: one copy of 48 x 4 x 2 x 3
// elements each, nine per tile.
__device__ __forceinline__ void issue_sources(const CUtensorMap *map, unsigned short *stage, unsigned long long *bar,
                                              int x0, int y0, const int zp[3]) {
    mbar_expect_tx(bar, STG_BYTES);
#pragma unroll 1
    for (int j = 0; j < 9; ++j) {
        const int ey = j % 3, ez = j / 3;
        // populations 3j .. 3j + 2: x from x0 - 8, rows from y0 - xi_y, planes from zp[ez]
        tma_load_4d(stage + 3 * j * STG_BOX, map, x0 - 8, y0 - (ey - 1), zp[ez], 3 * j, bar);
    }
}

// A tile at a periodic x / y edge: fetch the elements the copies filled with
// zeros (the consumer threads; the caller synchronises them afterwards).
template <int ST>
__device__ __forceinline__ void patch_edges(const Geom &g, const typename Codec<ST>::T *__restrict__ src,
                                            unsigned short *stage, int x0, int y0, const int zp[3]) {
    const int nx = g.nx, ny = g.ny, plane = (int)g.plane, ncell = (int)g.ncell;
    const unsigned short *raw = reinterpret_cast<const unsigned short *>(src);
    const int t = threadIdx.x;  // consumer thread 0 .. STG_CONS - 1
    if (x0 == 0 || x0 + STG_TX == nx) {
        // column 7 (x0 - 1) of the xi_x = +1 boxes at x0 = 0, column 40
        // (x0 + 32) of the xi_x = -1 boxes at the far edge: 9 boxes x 8 rows
        for (int k = t; k < 2 * 9 * STG_TY * STG_TZ; k += STG_TX * STG_TY) {
            const int side = k / (9 * STG_TY * STG_TZ), rest = k % (9 * STG_TY * STG_TZ);
            if (side == 0 ? x0 != 0 : x0 + STG_TX != nx) continue;
            const int b = rest / (STG_TY * STG_TZ), row = rest % (STG_TY * STG_TZ);
            const int ex = side == 0 ? 2 : 0, ey = b % 3, ez = b / 3, i = ex + 3 * ey + 9 * ez;
            const int r = row % STG_TY, zz = row / STG_TY;
            const int col = side == 0 ? 7 : STG_TX + 8;
            const int gx = side == 0 ? nx - 1 : 0;
            const int gy = wrap(y0 + r - (ey - 1), ny);
            stage[i * STG_BOX + (zz * STG_TY + r) * STG_BX + col] =
                raw[(size_t)i * ncell + (zp[ez] + zz) * plane + gy * nx + gx];
        }
    }
    if (y0 == 0 || y0 + STG_TY == ny) {
        // row 0 (y0 - 1) of the xi_y = +1 boxes at y0 = 0, row 3 (y0 + 4) of
        // the xi_y = -1 boxes at the far edge: 9 boxes x 2 planes x 34 columns
        constexpr int W = STG_TX + 2;
        for (int k = t; k < 2 * 9 * STG_TZ * W; k += STG_TX * STG_TY) {
            const int side = k / (9 * STG_TZ * W), rest = k % (9 * STG_TZ * W);
            if (side == 0 ? y0 != 0 : y0 + STG_TY != ny) continue;
            const int b = rest / (STG_TZ * W), rc = rest % (STG_TZ * W);
            const int ey = side == 0 ? 2 : 0, ex = b % 3, ez = b / 3, i = ex + 3 * ey + 9 * ez;
            const int zz = rc / W, col = 7 + rc % W;
            const int r = side == 0 ? 0 : STG_TY - 1;
            const int gx = wrap(x0 - 8 + col, nx);
            const int gy = side == 0 ? ny - 1 : 0;
            stage[i * STG_BOX + (zz * STG_TY + r) * STG_BX + col] =
                raw[(size_t)i * ncell + (zp[ez] + zz) * plane + gy * nx + gx];
        }
    }
}

// Bounded wait for the phase `parity` of an mbarrier (every thread).
__device__ __forceinline__ bool wait_bounded(unsigned long long *bar, unsigned parity) {
    bool done = false;
    for (unsigned it = 0; it < STG_WAIT_LIMIT && !done; ++it) done = mbar_try_wait(bar, parity);
    return done;
}

// The plain pull and stores for a tile the pipeline does not stage (kept out
// of line, so that the staged path's register allocation is its own).
template <int ST, int MODE>
__device__ __noinline__ void plain_pair(const Geom &g, const typename Codec<ST>::T *__restrict__ src,
                                        typename Codec<ST>::T *__restrict__ dst, const float *__restrict__ utop_in,
                                        float *__restrict__ utop_out, const BodySlot &S, const float *__restrict__ hbox,
                                        const BoxGeom &box, int x, int y, int z0) {
    k1_pair<ST, MODE>(g, src, dst, utop_in, utop_out, S, hbox, box, x, y, z0);
}

// Producer: one thread of the last warp.  Fills the input stage of tile t
// (the source copies of a staged tile; a plain arrival otherwise), and stores
// each computed output tile, in tile order.
template <int MODE>
__device__ __forceinline__ void produce(const CUtensorMap *lmap, const CUtensorMap *smap, const Geom &g,
                                        const BodySlot &S, const BoxGeom &box, DevState *st, int x0, int y0, int zb,
                                        int ntile, unsigned short *in, unsigned short *out, unsigned long long *full,
                                        unsigned long long *empty, unsigned long long *ofull,
                                        unsigned long long *oempty) {
    int fills[STG_NS] = {};
    auto fill = [&](int t) {
        const int s = t % STG_NS;
        int zp[3];
        if (tile_staged<MODE>(g, S, box, x0, y0, zb + STG_TZ * t, zp))
            issue_sources(lmap, in + s * 27 * STG_BOX, &full[s], x0, y0, zp);
        else
            mbar_arrive(&full[s]);
        fills[s] += 1;
    };
    for (int t = 0; t < STG_NS && t < ntile; ++t) fill(t);
    bool ok = true;
    for (int k = 0; k < ntile && ok; ++k) {
        const int b = k % STG_NO;
        ok = wait_bounded(&ofull[b], (k / STG_NO) & 1);
        if (!ok) break;
        int zp[3];
        if (tile_staged<MODE>(g, S, box, x0, y0, zb + STG_TZ * k, zp)) {
            tma_store_4d(smap, out + b * 27 * STG_OBOX, x0, y0, zp[1], 0);  // all 27 populations
            bulk_commit();
            bulk_wait_read();
        }
        mbar_arrive(&oempty[b]);
        const int t = k + STG_NS;
        if (t < ntile) {
            ok = wait_bounded(&empty[t % STG_NS], ((t / STG_NS) - 1) & 1);
            if (ok) fill(t);
        }
    }
    if (!ok) {
        // a wait ran out: latch the status and wait (bounded) for the copies
        // still in flight into the stages before the block's memory is released
        atomicCAS(&st->status, 0, STAT_TIMEOUT);
        for (int s = 0; s < STG_NS; ++s)
            if (fills[s] > 0) wait_bounded(&full[s], (fills[s] - 1) & 1);
    }
    bulk_wait_all();
}

// MODE: K1_ALL (whole window, no forcing; slot_out >= 0 carries the window
// slot) or K1_FAR (cells outside the near region of a coupled step).  Grid
// (nx / 32, ny / 4, ceil(nz / (2 STG_TPB))) blocks of STG_CONS + 32 threads
// and STG_SMEM bytes of dynamic shared memory.  lmap: source tensor map (box
// 48 x 4 x 2 x 3) of src; smap: destination tensor map (box 32 x 4 x 2 x 27)
// of dst.  Warps 0-3 compute the tiles (thread (tx, ty) = (lane, warp): the
// cell pair (x0 + tx, y0 + ty, z0 / z0 + 1)), warp 4 moves the data.
template <int ST, int MODE>
__global__ void __launch_bounds__(STG_CONS + 32, 3)
    k_collide_staged(const __grid_constant__ CUtensorMap lmap, const __grid_constant__ CUtensorMap smap, Geom g,
                     const typename Codec<ST>::T *__restrict__ src, typename Codec<ST>::T *__restrict__ dst,
                     const float *__restrict__ utop_in, float *__restrict__ utop_out, DevState *st, int slot,
                     int slot_out, const float *__restrict__ hbox, BoxGeom box) {
    extern __shared__ __align__(128) unsigned char stg_smem[];
    unsigned short *in = reinterpret_cast<unsigned short *>(stg_smem);  // [STG_NS][27][STG_BOX] sources
    unsigned short *out = in + STG_NS * 27 * STG_BOX;                     // [STG_NO][27][STG_OBOX] results
    unsigned long long *full = reinterpret_cast<unsigned long long *>(out + STG_NO * 27 * STG_OBOX);
    unsigned long long *empty = full + STG_NS, *ofull = empty + STG_NS, *oempty = ofull + STG_NO;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (MODE == K1_ALL && slot_out >= 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 &&
        threadIdx.x == 0) {
        st->s[slot_out] = st->s[slot];
        st->s[slot_out].reseed = -1;
        st->s[slot_out].step += 1;
    }
    const BodySlot &S = st->s[slot];
    const int x0 = blockIdx.x * STG_TX, y0 = blockIdx.y * STG_TY, zb = blockIdx.z * (STG_TZ * STG_TPB);
    const int ntile = min(STG_TPB, (g.nz - zb + STG_TZ - 1) / STG_TZ);
    if (threadIdx.x == 0) {
        for (int s = 0; s < STG_NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], STG_TY);  // one arrival per consumer warp
        }
        for (int b = 0; b < STG_NO; ++b) {
            mbar_init(&ofull[b], STG_TY);
            mbar_init(&oempty[b], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == STG_TY) {
        if (lane == 0) produce<MODE>(&lmap, &smap, g, S, box, st, x0, y0, zb, ntile, in, out, full, empty, ofull, oempty);
        return;
    }
    const int tx = lane, ty = warp, x = x0 + tx, y = y0 + ty;
    const bool edge = x0 == 0 || x0 + STG_TX == g.nx || y0 == 0 || y0 + STG_TY == g.ny;
#pragma unroll 1
    for (int k = 0; k < ntile; ++k) {
        const int s = k % STG_NS, b = k % STG_NO, z0 = zb + STG_TZ * k;
        int zp[3];
        const bool staged = tile_staged<MODE>(g, S, box, x0, y0, z0, zp);
        if (!wait_bounded(&full[s], (k / STG_NS) & 1)) return;  // the producer latches the timeout
        unsigned short *stage = in + s * 27 * STG_BOX;
        f2 q[27];
        if (staged) {
            if (edge) {
                patch_edges<ST>(g, src, stage, x0, y0, zp);
                fence_proxy_async();
                consumers_sync();
            }
            // population i: column tx + 8 - xi_x, row ty, plane 0 / 1 of box i
            const unsigned short *base = stage + ty * STG_BX + tx + 8;
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const unsigned short *pi = base + i * STG_BOX - (i % 3 - 1);
                q[i].x = from_bits<ST>(pi[0]);
                q[i].y = from_bits<ST>(pi[STG_TY * STG_BX]);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
        if (!staged) plain_pair<ST, MODE>(g, src, dst, utop_in, utop_out, S, hbox, box, x, y, z0);
        else {
            const int z[2] = {z0, z0 + 1};
            const bool on[2] = {true, true};
            k1_pair_collide_store<ST, MODE, false>(g, dst, utop_out, S, hbox, box, x, y, z, on, q);
        }
        // the output tile of this parity is free once the store of tile k - 2 read it
        if (k >= STG_NO && !wait_bounded(&oempty[b], ((k / STG_NO) - 1) & 1)) return;
        if (staged) {
            unsigned short *o = out + b * 27 * STG_OBOX + ty * STG_TX + tx;
            if (ST == ST_BF16 && g.sround) {
                // the random bits of every other path (sr_bits of the element;
                // planes z0 and z0 + 1 are zp[1] and zp[0])
                const int own_a = zp[1] * (int)g.plane + y * g.nx + x, own_b = zp[0] * (int)g.plane + y * g.nx + x;
                const int ncell = (int)g.ncell;
#pragma unroll
                for (int i = 0; i < 27; ++i) {
                    o[i * STG_OBOX] = bf16_sr_bits(q[i].x, sr_bits(i * ncell + own_a, S.step));
                    o[i * STG_OBOX + STG_TY * STG_TX] = bf16_sr_bits(q[i].y, sr_bits(i * ncell + own_b, S.step));
                }
            } else {
#pragma unroll
                for (int i = 0; i < 27; ++i) {
                    o[i * STG_OBOX] = to_bits<ST>(q[i].x);
                    o[i * STG_OBOX + STG_TY * STG_TX] = to_bits<ST>(q[i].y);
                }
            }
            fence_proxy_async();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ofull[b]);
    }
}

// ---------------------------------------------------------------------------
// Host side.

bool staged_eligible(const Geom &g, int storage) {
    return (storage == ST_F16 || storage == ST_BF16) && g.nx % STG_TX == 0 && g.ny % STG_TY == 0 &&
           g.nz % STG_TZ == 0 && g.nz >= 4;
}

// The 4-D tensor map (x, y, z, population) of one population buffer: source
// boxes (48 x 4 x 2 x 3: three populations) or destination boxes (32 x 4 x 2
// x 27: the whole output tile).  Returns false when the driver refuses it.
bool encode_population_map(CUtensorMap *map, const void *buf, const Geom &g, bool source) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 27};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 2, (cuuint64_t)g.plane * 2, (cuuint64_t)g.ncell * 2};
    const cuuint32_t boxdim[4] = {(cuuint32_t)(source ? STG_BX : STG_TX), STG_TY, STG_TZ, source ? 3u : 27u};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void *>(buf), dims, strides, boxdim,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Opt the staged kernels into their dynamic shared memory (current device).
bool prepare_staged() {
    const void *fns[4] = {(const void *)k_collide_staged<ST_F16, K1_FAR>, (const void *)k_collide_staged<ST_F16, K1_ALL>,
                          (const void *)k_collide_staged<ST_BF16, K1_FAR>,
                          (const void *)k_collide_staged<ST_BF16, K1_ALL>};
    for (const void *f : fns)
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)STG_SMEM) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    return true;
}

bool is_staged_kernel(const void *fn) {
    return fn == (const void *)k_collide_staged<ST_F16, K1_FAR> || fn == (const void *)k_collide_staged<ST_F16, K1_ALL> ||
           fn == (const void *)k_collide_staged<ST_BF16, K1_FAR> || fn == (const void *)k_collide_staged<ST_BF16, K1_ALL>;
}

cudaError_t launch_collide_staged(const Geom &g, int storage, const CUtensorMap &lmap, const CUtensorMap &smap,
                                  const void *src, void *dst, const float *utop_in, float *utop_out, DevState *st,
                                  int slot, int slot_out, const float *hbox, const BoxGeom &box, int region,
                                  cudaStream_t s) {
    const dim3 grid(g.nx / STG_TX, g.ny / STG_TY, (g.nz + STG_TZ * STG_TPB - 1) / (STG_TZ * STG_TPB));
    const dim3 blk(STG_CONS + 32);
    if (storage == ST_F16) {
        using T = __half;
        if (region == REGION_FAR)
            k_collide_staged<ST_F16, K1_FAR><<<grid, blk, STG_SMEM, s>>>(lmap, smap, g, (const T *)src, (T *)dst, utop_in,
                                                                         utop_out, st, slot, -1, hbox, box);
        else
            k_collide_staged<ST_F16, K1_ALL><<<grid, blk, STG_SMEM, s>>>(lmap, smap, g, (const T *)src, (T *)dst, utop_in,
                                                                         utop_out, st, slot, slot_out, hbox, box);
    } else {
        using T = __nv_bfloat16;
        if (region == REGION_FAR)
            k_collide_staged<ST_BF16, K1_FAR><<<grid, blk, STG_SMEM, s>>>(lmap, smap, g, (const T *)src, (T *)dst,
                                                                          utop_in, utop_out, st, slot, -1, hbox, box);
        else
            k_collide_staged<ST_BF16, K1_ALL><<<grid, blk, STG_SMEM, s>>>(
                lmap, smap, g, (const T *)src, (T *)dst, utop_in, utop_out, st, slot, slot_out, hbox, box);
    }
    return cudaGetLastError();
}

}  // namespace turret
