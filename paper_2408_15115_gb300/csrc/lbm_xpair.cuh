// lbm_xpair.cuh -- collide+stream of 16-bit population storage on pairs of
// x-adjacent cells, every population moved with 4-byte accesses (shared by the
// single-window kernel of lbm_xpair.cu and the batched bulk launch).
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
// word per population (BF16 with stochastic rounding: one hash per population
// serves the pair, as sr_bits defines it).  The arithmetic is the lane-generic collision, so a
// cell gets the bits it gets on any other path.
#pragma once
#include "lbm_cell.cuh"

namespace turret {

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

// Whether the tile [x0, x0 + tw) x [y0, y0 + th) x {z0, z0 + 1} (tw even)
// can run on x-pairs: inside the window (EXTENT: checked here; otherwise the
// launch guarantees it), every source on an interior plane other than the one
// entering the ring window, no closed x / y face met, and (MODE K1_FAR) no
// cell of the near region.
template <int MODE, bool EXTENT>
__device__ __forceinline__ bool xpair_tile_ok(const Geom &g, const BodySlot &S, const BoxGeom &box, int x0, int y0,
                                              int z0, int tw, int th) {
    bool ok = z0 >= 1 && z0 + 3 <= g.nz;
    if (EXTENT) ok = ok && (g.nx & 1) == 0 && x0 + tw <= g.nx && y0 + th <= g.ny;
#pragma unroll
    for (int zs = -1; zs <= 2; ++zs) ok = ok && zphys(z0 + zs, S.ring, g.nz) != S.reseed;
    if (g.bc_x != BC_PERIODIC && (x0 == 0 || x0 + tw == g.nx)) ok = false;
    if (g.bc_y != BC_PERIODIC && (y0 == 0 || y0 + th == g.ny)) ok = false;
    if (MODE == K1_FAR && ok)
        ok = !(xp_meets_near(x0, tw, S.box_lo[0], S.box_lo_w[0], box.Bx + 2 * NEAR_GROW, g.nx, g.bc_x == BC_PERIODIC) &&
               xp_meets_near(y0, th, S.box_lo[1], S.box_lo_w[1], box.By + 2 * NEAR_GROW, g.ny, g.bc_y == BC_PERIODIC) &&
               xp_meets_near(z0, 2, S.box_lo[2], S.box_lo_w[2], box.Bz + 2 * NEAR_GROW, g.nz,
                             g.bc_bottom == BC_PERIODIC));
    return ok;
}

// Collide+stream of the cells (x, y, zl) and (x + 1, y, zl) of a tile that
// xpair_tile_ok admits (x even; MODE K1_ALL or K1_FAR, no forcing).
template <int ST, int MODE>
__device__ __forceinline__ void xpair_cells(const Geom &g, const typename Codec<ST>::T *__restrict__ src,
                                            typename Codec<ST>::T *__restrict__ dst, float *__restrict__ utop_out,
                                            const BodySlot &S, const float *__restrict__ hbox, const BoxGeom &box,
                                            int x, int y, int zl) {
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
    if (ST == ST_BF16 && g.sround) {
        // one hash per population serves the pair (sr_bits: low half x, high half x + 1)
        const int own = zphys(zl, S.ring, g.nz) * plane + y * nx + x;  // even
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const unsigned h = pcg_hash(sr_key(i * ncell + own, S.step));
            d[(size_t)i * (ncell / 2)] =
                (unsigned)bf16_sr_bits(q[i].x, h & 0xffffu) | ((unsigned)bf16_sr_bits(q[i].y, h >> 16) << 16);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 27; ++i) d[(size_t)i * (ncell / 2)] = pack2<ST>(q[i]);
}

}  // namespace turret
