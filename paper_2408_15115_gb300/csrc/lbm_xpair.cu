// lbm_xpair.cu -- the single-window bulk collide+stream with 16-bit population
// storage on pairs of x-adjacent cells (lbm_xpair.cuh).
//
// A block of 32 x 4 threads owns a tile of 64 x 2 x 2 cells: a warp covers 64
// contiguous cells of one row (128-byte accesses), thread (tx, ty) the pair
// (x0 + 2 tx, x0 + 2 tx + 1) of row y0 + (ty & 1), plane z0 + (ty >> 1).
// Tiles that xpair_tile_ok admits take the x-pair path; the others (the
// boundary planes, the plane entering the ring window, closed x / y faces
// and, for far-cell launches, the near region) run the one-cell code over the
// same cells (thread t: column t of the tile's 128, both planes).  Both are
// the same arithmetic (and, with stochastic rounding, the same random bits),
// so results are bitwise equal to the plain kernel.
#include "lbm_xpair.cuh"

namespace turret {

namespace {

constexpr int XP_TX = 64, XP_TY = 2, XP_TZ = 2;  // cells per tile: 32 x 4 threads, one pair each

}  // namespace

// MODE: K1_ALL (whole window, no forcing; slot_out >= 0 carries the window
// slot) or K1_FAR (cells outside the near region of a coupled step).  Grid
// (nx / 64, ny / 2, nz / 2) blocks of 32 x 4 threads.
template <int ST, int MODE>
__global__ void __launch_bounds__(128, 5)
    k_collide_xpair(Geom g, const typename Codec<ST>::T *__restrict__ src, typename Codec<ST>::T *__restrict__ dst,
                    const float *__restrict__ utop_in, float *__restrict__ utop_out, DevState *st, int slot,
                    int slot_out, const float *__restrict__ hbox, BoxGeom box) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (MODE == K1_ALL && slot_out >= 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && tx == 0 &&
        ty == 0) {
        st->s[slot_out] = st->s[slot];
        st->s[slot_out].reseed = -1;
        st->s[slot_out].step += 1;
    }
    const BodySlot &S = st->s[slot];
    const int x0 = blockIdx.x * XP_TX, y0 = blockIdx.y * XP_TY, z0 = XP_TZ * blockIdx.z;
    if (!xpair_tile_ok<MODE, false>(g, S, box, x0, y0, z0, XP_TX, XP_TY)) {
        // the one-cell path: thread t takes column t of the tile, both planes.
        // Inline and scalar: as an out-of-line call the whole kernel measured
        // 12 % slower, with the cell-pair code inline 9 % slower (its register
        // use shapes the x-pair path's allocation).
        const int t = ty * 32 + tx;
        k1_cell<ST, MODE>(g, src, dst, utop_in, utop_out, S, hbox, box, x0 + t % XP_TX, y0 + t / XP_TX, z0);
        k1_cell<ST, MODE>(g, src, dst, utop_in, utop_out, S, hbox, box, x0 + t % XP_TX, y0 + t / XP_TX, z0 + 1);
        return;
    }
    xpair_cells<ST, MODE>(g, src, dst, utop_out, S, hbox, box, x0 + 2 * tx, y0 + (ty & 1), z0 + (ty >> 1));
}

// ---------------------------------------------------------------------------
// Host side.

bool xpair_eligible(const Geom &g, int storage) {
    return (storage == ST_F16 || storage == ST_BF16) && g.nx % XP_TX == 0 && g.ny % XP_TY == 0 &&
           g.nz % XP_TZ == 0 && g.nz >= 4;
}

cudaError_t launch_collide_xpair(const Geom &g, int storage, const void *src, void *dst, const float *utop_in,
                                 float *utop_out, DevState *st, int slot, int slot_out, const float *hbox,
                                 const BoxGeom &box, int region, cudaStream_t s) {
    const dim3 grid(g.nx / XP_TX, g.ny / XP_TY, g.nz / XP_TZ), blk(32, 4);
    if (storage == ST_F16) {
        using T = __half;
        if (region == REGION_FAR)
            k_collide_xpair<ST_F16, K1_FAR><<<grid, blk, 0, s>>>(g, (const T *)src, (T *)dst, utop_in, utop_out, st,
                                                                 slot, -1, hbox, box);
        else
            k_collide_xpair<ST_F16, K1_ALL><<<grid, blk, 0, s>>>(g, (const T *)src, (T *)dst, utop_in, utop_out, st,
                                                                 slot, slot_out, hbox, box);
    } else {
        using T = __nv_bfloat16;
        if (region == REGION_FAR)
            k_collide_xpair<ST_BF16, K1_FAR><<<grid, blk, 0, s>>>(g, (const T *)src, (T *)dst, utop_in, utop_out,
                                                                  st, slot, -1, hbox, box);
        else
            k_collide_xpair<ST_BF16, K1_ALL><<<grid, blk, 0, s>>>(g, (const T *)src, (T *)dst, utop_in, utop_out,
                                                                  st, slot, slot_out, hbox, box);
    }
    return cudaGetLastError();
}

bool is_xpair_kernel(const void *fn) {
    return fn == (const void *)k_collide_xpair<ST_F16, K1_FAR> || fn == (const void *)k_collide_xpair<ST_F16, K1_ALL> ||
           fn == (const void *)k_collide_xpair<ST_BF16, K1_FAR> || fn == (const void *)k_collide_xpair<ST_BF16, K1_ALL>;
}

}  // namespace turret
