// support_moments.cuh -- block code of the support-box moments and of the
// marker binning that feeds the immersed-boundary transfers (one launch in the
// single-run and the batched steps); the pull and moment code is the
// collide+stream's (lbm_cell.cuh), so both see identical populations.
#pragma once
#include "lbm_cell.cuh"

namespace turret {

// K2 + binning, one launch.  Blocks [0, nmom): u* and the stress of Eq. 10,
// sigma = -p I + (1/(2 tau) - 1) P1 with p = c_s^2 (rho - 1), at every
// support-box cell, from f(t+1) pulled from the post-collision buffer (box
// cells outside a closed face get zeros; cells no stencil reads, the outer
// layer among them, are skipped).  Blocks [nmom, nmom + ntiles): for
// one TILE^3 tile of the box, two lists in marker order (ordered compaction
// with warp ballots; no atomics): list 0, the markers whose 4x4x4 stencil
// overlaps the tile (spreading); list 1, those whose stencil overlaps the
// stencil of any marker based in the tile (rows of A).
constexpr int MB_THREADS = 128;

template <int ST>
__device__ __forceinline__ void mb_block(const Geom &g, const typename Codec<ST>::T *__restrict__ src,
                                         const float *__restrict__ utop_in, const DevState *__restrict__ st, int slot,
                                         const BoxGeom &box, const BoxArrays &ba, int nmom, int nm,
                                         const int *__restrict__ mbase, const int *__restrict__ mseg,
                                         int *__restrict__ tile_list, int *__restrict__ tile_count, int cap,
                                         DevState *stw, float rmin,
                                         float rmax, int blk) {
    if (blk >= nmom) {
        constexpr int NW = MB_THREADS / 32;
        const int tile = blk - nmom;
        const int tx = tile % box.tx, ty = (tile / box.tx) % box.ty, tz = tile / (box.tx * box.ty);
        const int t0[3] = {TILE * tx, TILE * ty, TILE * tz};
        {
            // Both lists hold markers whose stencil base b lies in [t0 - 3, t0 + 6]
            // per axis, i.e. whose position X lies in [t0 - 2, t0 + 8).  Markers
            // sit at rmin <= |X - C| <= rmax (body-frame radii, up to rounding):
            // a region outside that shell has no candidates.
            const BodySlot &S = st->s[slot];
            float dmin2 = 0.0f, dmax2 = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float c = (float)(S.Ci[a] - S.box_lo[a]) + (float)S.Cf[a];
                const float lo = (float)(t0[a] - 2), hi = (float)(t0[a] + 8);
                const float dn = fmaxf(fmaxf(lo - c, c - hi), 0.0f);
                const float dx = fmaxf(fabsf(c - lo), fabsf(c - hi));
                dmin2 += dn * dn;
                dmax2 += dx * dx;
            }
            const float margin = 0.25f;
            if (dmin2 > (rmax + margin) * (rmax + margin) ||
                (rmin > margin && dmax2 < (rmin - margin) * (rmin - margin))) {
                if (threadIdx.x < 2) tile_count[threadIdx.x * (box.tx * box.ty * box.tz) + tile] = 0;
                return;
            }
        }
        // CU chunks of MB_THREADS markers per pass: their loads are issued
        // together and their hits compacted chunk after chunk (marker order);
        // one barrier per pass, the warp counts alternating between two buffers
        constexpr int CU = 4;
        __shared__ int wcount[2][CU][2][NW];
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        const int nseg = (nm + MARKER_SEG - 1) / MARKER_SEG;
        int tot[2] = {0, 0};  // identical in every thread
        int par = 0;
        for (int group = 0; group < nm; group += CU * MB_THREADS) {
            // skip chunks whose segments' stencil bases all miss [t0 - 3, t0 + 6];
            // the test is the same in every thread, so a group with no chunk
            // left is skipped whole, barrier included
            bool reach[CU], any = false;
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int chunk = group + u * MB_THREADS;
                reach[u] = false;
                for (int sg = chunk / MARKER_SEG; sg < nseg && sg * MARKER_SEG < chunk + MB_THREADS; ++sg) {
                    const int *bb = mseg + 6 * sg;
                    bool in = true;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        in = in && __ldg(bb + 3 + a) + 3 >= t0[a] && __ldg(bb + a) <= t0[a] + TILE + 2;
                    reach[u] = reach[u] || in;
                }
                any = any || reach[u];
            }
            if (!any) continue;
            int pb[CU];
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int k = group + u * MB_THREADS + tid;
                pb[u] = (reach[u] && k < nm) ? __ldg(mbase + k) : -1;  // culled chunks load nothing
            }
            unsigned bal[CU][2];
            bool hit[CU][2];
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                hit[u][0] = hit[u][1] = pb[u] >= 0;
                const int b[3] = {pb[u] & 1023, (pb[u] >> 10) & 1023, (pb[u] >> 20) & 1023};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const bool lo = b[a] + 3 >= t0[a];
                    hit[u][0] = hit[u][0] && lo && (b[a] <= t0[a] + TILE - 1);  // stencil overlaps the tile
                    hit[u][1] = hit[u][1] && lo && (b[a] <= t0[a] + TILE + 2);  // ... or a stencil based in it
                }
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    bal[u][l] = __ballot_sync(0xffffffffu, hit[u][l]);
                    if (lane == 0) wcount[par][u][l][warp] = __popc(bal[u][l]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < CU; ++u)
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    int off = tot[l], sum = 0;
                    for (int w = 0; w < NW; ++w) {
                        const int c = wcount[par][u][l][w];
                        off += (w < warp) ? c : 0;
                        sum += c;
                    }
                    if (hit[u][l]) {
                        const int pos = off + __popc(bal[u][l] & ((1u << lane) - 1u));
                        if (pos < cap)
                            tile_list[((size_t)l * (box.tx * box.ty * box.tz) + tile) * cap + pos] =
                                group + u * MB_THREADS + tid;
                    }
                    tot[l] += sum;
                }
            par ^= 1;
        }
        if (tid < 2) {
            tile_count[tid * (box.tx * box.ty * box.tz) + tile] = tot[tid] < cap ? tot[tid] : cap;
            if (tot[tid] > cap) atomicCAS(&stw->status, 0, STAT_OVERFLOW);
        }
        return;
    }
    const long long b = (long long)blk * blockDim.x + threadIdx.x;
    if (b >= box.nbox) return;
    const int bx = (int)(b % box.Bx);
    const int by = (int)((b / box.Bx) % box.By);
    const int bz = (int)(b / ((long long)box.Bx * box.By));
    // The outermost layer of the box is never read: along each axis a stencil
    // of a point P with |P_a - C_a| <= R = rmax + F_OFFSET covers cells
    // floor(C_a - R) - 1 .. floor(C_a + R) + 2, inside the box's
    // Ci - rc - 1 .. Ci + rc + 2 (rc = ceil R).  Skipping it keeps every pull
    // of this kernel inside the box, which is the near region: the moments
    // then depend on the near launch only, never on the far one.
    if (bx == 0 || by == 0 || bz == 0 || bx == box.Bx - 1 || by == box.By - 1 || bz == box.Bz - 1) return;
    {
        // The moments are read only inside the 4x4x4 stencils of the markers
        // (u*) and of the offset points X + F_OFFSET n (sigma, p).  Those points
        // lie at rmin - F_OFFSET <= |P - C| <= rmax + F_OFFSET, and a stencil
        // cell within 2 cells of P per axis (2 sqrt 3 in all): cells outside
        // that shell (the corners of the box, the core of a large body) are
        // never read and are skipped.
        const BodySlot &S = st->s[slot];
        const int bb[3] = {bx, by, bz};
        float d2 = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float d = (float)bb[a] - ((float)(S.Ci[a] - S.box_lo[a]) + (float)S.Cf[a]);
            d2 += d * d;
        }
        const float reach = F_OFFSET + 3.4641016f + 0.25f;
        if (d2 > (rmax + reach) * (rmax + reach) || (rmin > reach && d2 < (rmin - reach) * (rmin - reach))) return;
    }
    int c[3] = {st->s[slot].box_lo[0] + bx, st->s[slot].box_lo[1] + by, st->s[slot].box_lo[2] + bz};
    const int n[3] = {g.nx, g.ny, g.nz};
    const bool per[3] = {g.bc_x == BC_PERIODIC, g.bc_y == BC_PERIODIC, g.bc_bottom == BC_PERIODIC};
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (per[a]) {
            c[a] %= n[a];
            if (c[a] < 0) c[a] += n[a];
        } else if (c[a] < 0 || c[a] >= n[a]) {
            inside = false;
        }
    }
    if (!inside) {
#pragma unroll
        for (int k = 0; k < 3; ++k) ba.u[k * box.nbox + b] = 0.0f;
#pragma unroll
        for (int k = 0; k < 6; ++k) ba.s[k * box.nbox + b] = 0.0f;
        ba.p[b] = 0.0f;
        return;
    }
    float q[27];
    pull27<ST>(g, src, c[0], c[1], c[2], st->s[slot].ring, st->s[slot].reseed, utop_in, q);
    const MacroR<float> M = macro_raw<ST>(moments_raw<ST>(q));
    const float tau = tau_of(g, c[2]);
    // (1/(2 tau) - 1) P1 with P1 = P1~ / 216 = P / (216 K)
    const float k2 = (0.5f / tau - 1.0f) * (INV_SCALE / Codec<ST>::K);
    const float p = M.drho * (1.0f / 3.0f);
    ba.u[b] = M.ux;
    ba.u[box.nbox + b] = M.uy;
    ba.u[2 * box.nbox + b] = M.uz;
    ba.s[b] = -p + k2 * M.Pxx;
    ba.s[box.nbox + b] = -p + k2 * M.Pyy;
    ba.s[2 * box.nbox + b] = -p + k2 * M.Pzz;
    ba.s[3 * box.nbox + b] = k2 * M.Pxy;
    ba.s[4 * box.nbox + b] = k2 * M.Pxz;
    ba.s[5 * box.nbox + b] = k2 * M.Pyz;
    ba.p[b] = p;
}

}  // namespace turret
