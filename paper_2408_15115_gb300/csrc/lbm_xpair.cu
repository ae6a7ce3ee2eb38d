// lbm_xpair.cu -- the bulk collide+stream with 16-bit population storage on
// pairs of x-adjacent cells, every population moved with 4-byte accesses.
//
// With FP16 / BF16 storage, 2-byte global accesses stream at about 5 TB/s on
// this part whatever their alignment, while 4-byte accesses reach the copy
// bandwidth.  Here a thread owns the cells (x, x + 1) of one row (x even), and
// the packed f32x2 arithmetic of the collision runs over that pair instead of
// a (z, z + 1) pair.  Each population is read as aligned 4-byte words: the
// word at x for xi_x = 0; for xi_x = +1 the sources (x - 1, x) are the high
// half of the word at x - 2 and the low half of the word at x; for xi_x = -1
// the sources (x + 1, x + 2) are the high half of the word at x and the low
// half of the word at x + 2 (45 loads per pair, the extra words from the same
// cache lines as the neighbouring threads').  Results leave as one 4-byte
// word per population.
//
// A block of 32 x 4 threads owns a tile of 64 x 2 x 2 cells: a warp covers 64
// contiguous cells of one row (128-byte accesses), thread (tx, ty) the pair
// (x0 + 2 tx, x0 + 2 tx + 1) of row y0 + (ty & 1), plane z0 + (ty >> 1).
// Tiles whose sources all lie on interior planes,
// away from the plane entering the ring window, closed x / y faces and (far-
// cell launches) the near region take this path; the others run the one-cell
// code over the same cells (thread t: column t of the tile's 128, both
// planes).  Both are the same arithmetic
// (the lane-generic collision), so results are bitwise equal to the plain kernel.
// BF16 with stochastic rounding keeps the plain kernel: its random bits are
// keyed to the (z, z + 1) pairing.
#include "lbm_cell.cuh"

namespace turret {

namespace {

constexpr int XP_TX = 64, XP_TY = 2, XP_TZ = 2;  // cells per tile: 32 x 4 threads, one pair each

template <int ST>
__device__ __forceinline__ f2 unpack2(unsigned w);
template <>
__device__ __forceinline__ f2 unpack2<ST_F16>(unsigned w) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}
template <>
__device__ __forceinline__ f2 unpack2<ST_BF16>(unsigned w) {
    // a BF16 value is the high half of the FP32 value with the same bits
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

template <int ST>
__device__ __forceinline__ unsigned pack2(f2 v);
template <>
__device__ __forceinline__ unsigned pack2<ST_F16>(f2 v) {
    const __half2 h = __floats2half2_rn(v.x, v.y);  // each half rounded to nearest even
    return *reinterpret_cast<const unsigned *>(&h);
}
template <>
__device__ __forceinline__ unsigned pack2<ST_BF16>(f2 v) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    return *reinterpret_cast<const unsigned *>(&h);
}

__device__ __forceinline__ unsigned ld_word(const void *base, int elem) {
    return __ldg(reinterpret_cast<const unsigned *>(static_cast<const unsigned short *>(base) + elem));
}

// Whether the cells [c0, c0 + len) of one axis meet the near region (relative
// coordinates 0 .. ext - 1 from the support box origin less NEAR_GROW).
__device__ __forceinline__ bool xp_meets_near(int c0, int len, int lo, int lo_w, int ext, int n, bool periodic) {
    const int r0 = rel_axis(c0, lo, lo_w, NEAR_GROW, n, periodic);
    return periodic ? (r0 < ext || r0 + len > n) : (r0 < ext && r0 + len > 0);
}

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
    // block-uniform: sources on interior planes z0 - 1 .. z0 + 2, none of them
    // the entering plane, no closed face met, no near-region cell
    bool ok = z0 >= 1 && z0 + XP_TZ + 1 <= g.nz;
#pragma unroll
    for (int zs = -1; zs <= XP_TZ; ++zs) ok = ok && zphys(z0 + zs, S.ring, g.nz) != S.reseed;
    if (g.bc_x != BC_PERIODIC && (x0 == 0 || x0 + XP_TX == g.nx)) ok = false;
    if (g.bc_y != BC_PERIODIC && (y0 == 0 || y0 + XP_TY == g.ny)) ok = false;
    if (MODE == K1_FAR && ok)
        ok = !(xp_meets_near(x0, XP_TX, S.box_lo[0], S.box_lo_w[0], box.Bx + 2 * NEAR_GROW, g.nx,
                             g.bc_x == BC_PERIODIC) &&
               xp_meets_near(y0, XP_TY, S.box_lo[1], S.box_lo_w[1], box.By + 2 * NEAR_GROW, g.ny,
                             g.bc_y == BC_PERIODIC) &&
               xp_meets_near(z0, XP_TZ, S.box_lo[2], S.box_lo_w[2], box.Bz + 2 * NEAR_GROW, g.nz,
                             g.bc_bottom == BC_PERIODIC));
    if (!ok) {
        // the one-cell path: thread t takes column t of the tile, both planes.
        // Inline and scalar: as an out-of-line call the whole kernel measured
        // 12 % slower, with the cell-pair code inline 9 % slower (its register
        // use shapes the x-pair path's allocation).
        const int t = ty * 32 + tx;
        k1_cell<ST, MODE>(g, src, dst, utop_in, utop_out, S, hbox, box, x0 + t % XP_TX, y0 + t / XP_TX, z0);
        k1_cell<ST, MODE>(g, src, dst, utop_in, utop_out, S, hbox, box, x0 + t % XP_TX, y0 + t / XP_TX, z0 + 1);
        return;
    }
    const int x = x0 + 2 * tx, y = y0 + (ty & 1), zl = z0 + (ty >> 1);
    const int nx = g.nx, plane = (int)g.plane, ncell = (int)g.ncell;
    const int xm = x == 0 ? nx - 2 : x - 2, xp = x + 2 == nx ? 0 : x + 2;  // periodic here when at an edge
    int ys[3];
#pragma unroll
    for (int ey = 0; ey < 3; ++ey) {
        int yy = y - (ey - 1);
        yy += yy < 0 ? g.ny : 0;
        yy -= yy >= g.ny ? g.ny : 0;
        ys[ey] = yy * nx;
    }
    f2 q[27];
#pragma unroll
    for (int ez = 0; ez < 3; ++ez) {
        const int zrow = zphys(zl - (ez - 1), S.ring, g.nz) * plane;
#pragma unroll
        for (int ey = 0; ey < 3; ++ey) {
            const int row = zrow + ys[ey];
#pragma unroll
            for (int ex = 0; ex < 3; ++ex) {
                const int i = ex + 3 * ey + 9 * ez;
                const typename Codec<ST>::T *r = src + (size_t)i * ncell + row;
                const unsigned a = ld_word(r, x);
                unsigned w;
                if (ex == 1) w = a;
                else if (ex == 2) w = __byte_perm(ld_word(r, xm), a, 0x5432);  // (x - 1, x)
                else w = __byte_perm(a, ld_word(r, xp), 0x5432);                // (x + 1, x + 2)
                q[i] = unpack2<ST>(w);
            }
        }
    }
    // the pair shares its plane: the plane's relaxation time for both lanes
    const int z[2] = {zl, zl};
    const bool on[2] = {true, true};
    k1_pair_collide_store<ST, MODE, false>(g, dst, utop_out, S, hbox, box, x, y, z, on, q);
    unsigned *d = reinterpret_cast<unsigned *>(reinterpret_cast<unsigned short *>(dst) + zphys(zl, S.ring, g.nz) * plane +
                                               y * nx + x);
#pragma unroll
    for (int i = 0; i < 27; ++i) d[(size_t)i * (ncell / 2)] = pack2<ST>(q[i]);
}

// ---------------------------------------------------------------------------
// Host side.

bool xpair_eligible(const Geom &g, int storage) {
    return (storage == ST_F16 || (storage == ST_BF16 && !g.sround)) && g.nx % XP_TX == 0 && g.ny % XP_TY == 0 &&
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
