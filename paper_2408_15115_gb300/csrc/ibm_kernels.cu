// ibm_kernels.cu -- rigid-body update, marker kinematics and the
// immersed-boundary transfers of the Palabos Turret step (arXiv 2408.15115).
//
//   k_particle_markers : FP64 leap-frog 6DOF with the orientation
//                predictor-corrector (Sec. 2.3) and the vertical window slide,
//                spread over the lanes of warp 0 of every block (GB300 has
//                little FP64 throughput, so the path is short, lane-parallel
//                and free of division); then, in the same launch, the marker kinematics
//                X_k = C_m + M^T Xb_k, n_k = M^T nb_k, U_k = v + w x (X_k - C_m)
//                and each marker's 4x4x4 Peskin stencil (Sec. 2.2) in
//                support-box coordinates.
//   k_interp0_rows : I[u](X_k) = sum_x u(x) W(x - X_k) for u* and sigma, one
//                warp per marker, two stencil cells per lane, xor-shuffle sums
//                (deterministic); forms dS sigma.n and its moment about C_m
//                for the surface force (Sec. 2.2 end) and row k of the
//                interaction matrix A of the IBM cycles; one block per marker.
//   k_cycle    : one IBM cycle as h <- h + r0 - A h (a sparse product, one
//                warp per marker), equal to spreading h and interpolating
//                u* + S h without touching the grid.
//   k_reduce_ft: F and T summed in FP64 in a fixed order (one block); it runs
//                on its own graph branch, off the critical path of the cycles.
//   k_spread   : h_imm = S[h](x) = sum_k h_k W(x - X_k) dS_k as a gather: one block
//                per 4^3 tile of the support box stages the tile's candidate
//                records (built with the support-box moments, in marker order)
//                in shared memory; 8 slices of the candidates per cell, added
//                in slice order -- no atomics, bitwise reproducible.
#include <math.h>

#include "turret_internal.cuh"

namespace turret {

// Peskin 4-point kernel (Sec. 2.2) on its two branches, argument |r|.
__device__ __forceinline__ float peskin_in(float a) {
    return 0.125f * (3.0f - 2.0f * a + sqrtf(1.0f + 4.0f * a - 4.0f * a * a));
}
__device__ __forceinline__ float peskin_out(float a) {
    return 0.125f * (5.0f - 2.0f * a - sqrtf(fmaxf(0.0f, -7.0f + 12.0f * a - 4.0f * a * a)));
}

constexpr int PM_THREADS = MARKER_SEG;

// Every block recomputes the (tiny) rigid-body update from slot `slot` in
// warp 0 -- identical inputs, identical FP64 results -- and block 0 stores it
// in the other slot, so the marker work spreads over many SMs with no
// grid-wide wait.
__device__ __forceinline__ void pm_block(const Geom &g, const BodyConst &bc, const BoxGeom &box, DevState *st,
                                         int slot, int advance, const MarkerArrays &m, int blk) {
    __shared__ BodySlot S;  // the body at the markers' time level
    __shared__ double s_F[3], s_T[3], s_src[3], s_sb[3], s_wb[3], s_mid[9], s_dn[9];
    __shared__ float f_d[9], f_v[3], f_w[3], f_cf[3];
    __shared__ int i_ci[3], i_lo[3];
    const int tid = threadIdx.x;
    const int so = advance ? (slot ^ 1) : slot;  // slot of the markers' time level
    if (tid < 32) {
        const int lane = tid;
        {
            const int *gsrc = reinterpret_cast<const int *>(&st->s[slot]);
            int *sdst = reinterpret_cast<int *>(&S);
            for (int q = lane; q < (int)(sizeof(BodySlot) / 4); q += 32) sdst[q] = gsrc[q];
            if (lane < 3) {
                s_F[lane] = st->F[lane];
                s_T[lane] = st->T[lane];
            }
        }
        __syncwarp();
        if (advance) {
            // ---- 6DOF, Sec. 2.3 (dt = 1, rho_f = 1, m = kappa V) ------------------
            if (lane < 3) {
                // v(t+1/2), or 0 for a held centre
                S.v[lane] = bc.fixed ? 0.0 : S.v[lane] + bc.g_eff[lane] + s_F[lane] * bc.inv_mass;
                S.r[lane] += S.v[lane];                                 // r(t+1)
                if (bc.rot_form == 1) {
                    s_src[lane] = s_T[lane];
                } else {
                    S.L[lane] += s_T[lane];  // L(t+1/2) = L(t-1/2) + T(t)
                    s_src[lane] = S.L[lane];
                }
            }
            __syncwarp();
            if (lane < 3)  // body-frame components M src (M has rows d_i)
                s_sb[lane] = S.d[3 * lane] * s_src[0] + S.d[3 * lane + 1] * s_src[1] + S.d[3 * lane + 2] * s_src[2];
            __syncwarp();
            if (lane < 3)  // (J/m)^-1 / m, a host constant
                s_wb[lane] = bc.Jinv_b[3 * lane] * s_sb[0] + bc.Jinv_b[3 * lane + 1] * s_sb[1] +
                             bc.Jinv_b[3 * lane + 2] * s_sb[2];
            __syncwarp();
            if (lane < 3) {  // back to the lab frame: M^T wb
                const double wl = S.d[lane] * s_wb[0] + S.d[3 + lane] * s_wb[1] + S.d[6 + lane] * s_wb[2];
                S.w[lane] = (bc.rot_form == 1) ? S.w[lane] + wl : wl;
            }
            __syncwarp();
            // d_i^pred = d_i + w x d_i;  d_i(t+1) = d_i + w x (d_i + d_i^pred) / 2
            const int i = lane / 3, a = lane % 3, a1 = (a + 1) % 3, a2 = (a + 2) % 3;
            if (lane < 9) s_mid[lane] = S.d[lane] + 0.5 * (S.w[a1] * S.d[3 * i + a2] - S.w[a2] * S.d[3 * i + a1]);
            __syncwarp();
            if (lane < 9) s_dn[lane] = S.d[lane] + (S.w[a1] * s_mid[3 * i + a2] - S.w[a2] * s_mid[3 * i + a1]);
            __syncwarp();
            if (lane == 0) {
                for (int k = 0; k < 9; ++k) S.d[k] = s_dn[k];
                if (bc.renorm) {  // modified Gram-Schmidt of d_0, d_1, d_2
                    for (int q = 0; q < 3; ++q) {
                        for (int j = 0; j < q; ++j) {
                            double pj = 0.0;
                            for (int c = 0; c < 3; ++c) pj += S.d[3 * q + c] * S.d[3 * j + c];
                            for (int c = 0; c < 3; ++c) S.d[3 * q + c] -= pj * S.d[3 * j + c];
                        }
                        const double il = rsqrt(S.d[3 * q] * S.d[3 * q] + S.d[3 * q + 1] * S.d[3 * q + 1] +
                                                S.d[3 * q + 2] * S.d[3 * q + 2]);
                        for (int c = 0; c < 3; ++c) S.d[3 * q + c] *= il;
                    }
                }
                // vertical slide of the ring window: one plane per step at most
                int ring = S.ring;
                int reseed = -1;
                if (bc.slide) {
                    const double dz = (S.r[2] - (double)S.origin[2]) - bc.anchor_z;
                    if (dz <= -1.0) {
                        S.origin[2] -= 1;
                        ring = (ring == 0) ? g.nz - 1 : ring - 1;
                        reseed = ring;  // new logical bottom plane
                    } else if (dz >= 1.0) {
                        S.origin[2] += 1;
                        ring = (ring + 1 == g.nz) ? 0 : ring + 1;
                        reseed = (ring == 0) ? g.nz - 1 : ring - 1;  // new logical top plane
                    }
                }
                const int nn[3] = {g.nx, g.ny, g.nz};
                const bool pp[3] = {g.bc_x == BC_PERIODIC, g.bc_y == BC_PERIODIC, g.bc_bottom == BC_PERIODIC};
                for (int c = 0; c < 3; ++c) {
                    const double C = S.r[c] - (double)S.origin[c];
                    const double fl = floor(C);
                    S.Ci[c] = (int)fl;
                    S.Cf[c] = C - fl;
                    S.box_lo[c] = (int)fl - bc.rc - 2;
                    int lw = S.box_lo[c];
                    if (pp[c]) {
                        lw %= nn[c];
                        if (lw < 0) lw += nn[c];
                    }
                    S.box_lo_w[c] = lw;
                }
                S.ring = ring;
                S.reseed = reseed;
                S.step += 1;
            }
            __syncwarp();
            if (blk == 0 && lane < 8) st->pr.slip[lane] = 0u;
            if (blk == 0) {
                int *gdst = reinterpret_cast<int *>(&st->s[so]);
                const int *ssrc = reinterpret_cast<const int *>(&S);
                for (int q = lane; q < (int)(sizeof(BodySlot) / 4); q += 32) gdst[q] = ssrc[q];
            }
        }
        // marker velocities: v, w at t + 1/2 (the paper's step), or in the
        // predictor modes their estimates at t + 1 from the predicted force
        // and torque, v^ = v + (g_eff + F^ / m) / 2, L^ = L + T^ / 2 (or
        // w^ = w + (J/m)^-1 T^ / (2 m) in the literal rotation form)
        const bool pred = advance && bc.predictor != 0 && (bc.pred_opts & PRED_VEL) && st->pr.predicted;
        if (pred) {
            if (lane < 3) {
                s_src[lane] = st->pr.That[lane];
                s_F[lane] = bc.fixed ? 0.0 : S.v[lane] + 0.5 * (bc.g_eff[lane] + st->pr.Fhat[lane] * bc.inv_mass);
            }
            __syncwarp();
            if (lane < 3) {
                const double src = (bc.rot_form == 1) ? s_src[0] : S.L[0] + 0.5 * s_src[0];
                const double src1 = (bc.rot_form == 1) ? s_src[1] : S.L[1] + 0.5 * s_src[1];
                const double src2 = (bc.rot_form == 1) ? s_src[2] : S.L[2] + 0.5 * s_src[2];
                s_sb[lane] = S.d[3 * lane] * src + S.d[3 * lane + 1] * src1 + S.d[3 * lane + 2] * src2;
            }
            __syncwarp();
            if (lane < 3)
                s_wb[lane] = bc.Jinv_b[3 * lane] * s_sb[0] + bc.Jinv_b[3 * lane + 1] * s_sb[1] +
                             bc.Jinv_b[3 * lane + 2] * s_sb[2];
            __syncwarp();
            if (lane < 3) {
                const double wl = S.d[lane] * s_wb[0] + S.d[3 + lane] * s_wb[1] + S.d[6 + lane] * s_wb[2];
                s_T[lane] = (bc.rot_form == 1) ? S.w[lane] + 0.5 * wl : wl;
            }
            __syncwarp();
        }
        if (lane < 9) f_d[lane] = (float)S.d[lane];
        if (lane < 3) {
            f_v[lane] = (float)(pred ? s_F[lane] : S.v[lane]);
            f_w[lane] = (float)(pred ? s_T[lane] : S.w[lane]);
            f_cf[lane] = (float)S.Cf[lane];
            i_ci[lane] = S.Ci[lane];
            i_lo[lane] = S.box_lo[lane];
        }
    }
    __syncthreads();
    // ---- markers ---------------------------------------------------------------
    const int nm = bc.nm;
    const int n[3] = {g.nx, g.ny, g.nz};
    const bool per[3] = {g.bc_x == BC_PERIODIC, g.bc_y == BC_PERIODIC, g.bc_bottom == BC_PERIODIC};
    const int B[3] = {box.Bx, box.By, box.Bz};
    const int k = blk * PM_THREADS + tid;
    int bbv[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff};  // no marker: neutral for the minimum
    int bbmax[3] = {-1, -1, -1};
    if (k < nm) {
        bool bad = false;
        const float xb[3] = {m.Xb[k], m.Xb[nm + k], m.Xb[2 * nm + k]};
        const float nbv[3] = {m.nb[k], m.nb[nm + k], m.nb[2 * nm + k]};
        float arm[3], nn[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            arm[a] = f_d[a] * xb[0] + f_d[3 + a] * xb[1] + f_d[6 + a] * xb[2];
            nn[a] = f_d[a] * nbv[0] + f_d[3 + a] * nbv[1] + f_d[6 + a] * nbv[2];
        }
        const float U[3] = {f_v[0] + (f_w[1] * arm[2] - f_w[2] * arm[1]), f_v[1] + (f_w[2] * arm[0] - f_w[0] * arm[2]),
                            f_v[2] + (f_w[0] * arm[1] - f_w[1] * arm[0])};
        MRec r;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float xr = f_cf[a] + arm[a];  // marker position relative to Ci
            const float fl = floorf(xr);
            const float t = xr - fl;            // in [0, 1)
            int base_rel = (int)fl - 1;         // stencil cells base_rel .. base_rel + 3
            int bv = i_ci[a] + base_rel - i_lo[a];
            float w4[4] = {peskin_out(1.0f + t), peskin_in(t), peskin_in(1.0f - t), peskin_out(2.0f - t)};
            // a non-finite position, or a stencil reaching the box's outer layer
            // (never computed by the moments kernel), must never index memory or
            // read unset moments: park the stencil at the box origin with zero
            // weights and latch the status
            if (!isfinite(xr) || bv < 1 || bv > B[a] - 5) {
                bv = 0;
                base_rel = i_lo[a] - i_ci[a];
                w4[0] = w4[1] = w4[2] = w4[3] = 0.0f;
                bad = true;
            }
            const int abs_base = i_ci[a] + base_rel;
            if (!per[a] && (abs_base < 0 || abs_base + 3 > n[a] - 1)) bad = true;
            bbv[a] = bv;
            float *dstw = (a == 0) ? r.wx : (a == 1) ? r.wy : r.wz;
#pragma unroll
            for (int q = 0; q < 4; ++q) dstw[q] = w4[q];
            m.U[a * nm + k] = U[a];
            m.n[a * nm + k] = nn[a];
            m.arm[a * nm + k] = arm[a];
        }
        r.base = bbv[0] | (bbv[1] << 10) | (bbv[2] << 20);
        r.hdS[0] = r.hdS[1] = r.hdS[2] = 0.0f;
        m.rec[k] = r;
        m.base[k] = r.base;
        // the stencil of the point of the stress surface, X + F_OFFSET n
        // (force_eval 0; the marker's own stencil otherwise)
        if (bc.force_eval == 0) {
            MRec ro;
            int bo[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float xr = f_cf[a] + arm[a] + F_OFFSET * nn[a];
                const float fl = floorf(xr);
                const float t = xr - fl;
                int base_rel = (int)fl - 1;
                int bv = i_ci[a] + base_rel - i_lo[a];
                float w4[4] = {peskin_out(1.0f + t), peskin_in(t), peskin_in(1.0f - t), peskin_out(2.0f - t)};
                if (!isfinite(xr) || bv < 1 || bv > B[a] - 5) {
                    bv = 0;
                    base_rel = i_lo[a] - i_ci[a];
                    w4[0] = w4[1] = w4[2] = w4[3] = 0.0f;
                    bad = true;
                }
                const int abs_base = i_ci[a] + base_rel;
                if (!per[a] && (abs_base < 0 || abs_base + 3 > n[a] - 1)) bad = true;
                bo[a] = bv;
                float *dstw = (a == 0) ? ro.wx : (a == 1) ? ro.wy : ro.wz;
#pragma unroll
                for (int q = 0; q < 4; ++q) dstw[q] = w4[q];
            }
            ro.base = bo[0] | (bo[1] << 10) | (bo[2] << 20);
            ro.hdS[0] = ro.hdS[1] = ro.hdS[2] = 0.0f;
            m.reco[k] = ro;
        }
        if (bad) atomicCAS(&st->status, 0, STAT_DOMAIN);  // the first latched error wins
        for (int a = 0; a < 3; ++a) bbmax[a] = bbv[a];
    }
    // bounding box of the stencil bases of this block's markers (a segment of
    // PM_THREADS consecutive markers), read by the tile-list scan to skip
    // segments that cannot reach a tile
    __shared__ int s_seg[PM_THREADS / 32][6];
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int lo = __reduce_min_sync(0xffffffffu, bbv[a]);
        const int hi = __reduce_max_sync(0xffffffffu, bbmax[a]);
        if (lane == 0) {
            s_seg[warp][a] = lo;
            s_seg[warp][3 + a] = hi;
        }
    }
    __syncthreads();
    if (tid < 6) {
        int v = s_seg[0][tid];
        for (int w = 1; w < PM_THREADS / 32; ++w) v = (tid < 3) ? min(v, s_seg[w][tid]) : max(v, s_seg[w][tid]);
        m.seg[blk * 6 + tid] = v;
    }
}

__global__ void __launch_bounds__(PM_THREADS) k_particle_markers(Geom g, BodyConst bc, BoxGeom box, DevState *st,
                                                                  int slot, int advance, MarkerArrays m) {
    pm_block(g, bc, box, st, slot, advance, m, blockIdx.x);
}

__device__ __forceinline__ float pick4(const float w[4], int i) {
    return i == 0 ? w[0] : (i == 1 ? w[1] : (i == 2 ? w[2] : w[3]));
}

// Overlap of two 1-D 4-point stencils whose bases differ by d (|d| <= 3):
// sum_c wk[c - bk] wj[c - bj] over the common cells.
__device__ __forceinline__ float overlap4(const float wk[4], const float wj[4], int d) {
    float o = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int ii = i - d;
        if (ii >= 0 && ii < 4) o = fmaf(wk[i], pick4(wj, ii), o);
    }
    return o;
}

// Step l = 0 of Sec. 2.2 plus the operator of steps l = 1..3 in matrix form.
// Interpolating u* + S[h] at X_k gives I[u*]_k + sum_j A_kj h_j with
// A_kj = dS_j sum_x W(x - X_k) W(x - X_j); the Peskin weight is a tensor
// product, so A_kj = dS_j Ox Oy Oz with one 4-point overlap per axis.
// One block per marker k:
//   warp 0: interpolation of u* and sigma (two stencil cells per lane,
//           xor-shuffle sums), h^0 = U - I[u*], the traction dS sigma.n and
//           its moment about C_m;
//   all   : row k of A from the candidate list of the tile holding k's stencil
//           base, one candidate per thread, block-wide ordered compaction in
//           list (= marker) order: reproducible.
constexpr int ROWS_THREADS = 256;
constexpr int ROWS_WARPS = ROWS_THREADS / 32;

// Step l = 0 for marker k by one warp: interpolation of u* and sigma (two
// stencil cells per lane, xor-shuffle sums), h^0 = U - I[u*] and the
// traction dS sigma.n with its moment about C_m.
// warm: the IBM cycles start from the previous step's h (kept in hl).
// Two stencil cells of a 4x4x4 stencil per lane: the cell offsets and weights.
__device__ __forceinline__ void lane_cells(const BoxGeom &box, const MRec &r, int lane, size_t &c0, size_t &c1,
                                           float &w0, float &w1) {
    const int bx = r.base & 1023, by = (r.base >> 10) & 1023, bz = (r.base >> 20) & 1023;
    const int i = lane & 3, j = (lane >> 2) & 3, kz = lane >> 4;
    const float wxy = pick4(r.wx, i) * pick4(r.wy, j);
    w0 = wxy * (kz ? r.wz[1] : r.wz[0]);
    w1 = wxy * (kz ? r.wz[3] : r.wz[2]);
    c0 = ((size_t)(bz + kz) * box.By + (by + j)) * box.Bx + (bx + i);
    c1 = c0 + 2 * (size_t)box.By * box.Bx;
}

// m.force_eval 0: the stress at the point X + F_OFFSET n of the offset
// surface, with its area and arm; 1: at the marker, as printed
__device__ __forceinline__ void interp_marker_warp(const BoxGeom &box, int nm, const MarkerArrays &m,
                                                   const BoxArrays &ba, int k, const MRec &rk, int lane, int warm) {
    const int fe = m.force_eval;
    size_t c0, c1, d0, d1;
    float w0, w1, v0, v1;
    lane_cells(box, rk, lane, c0, c1, w0, w1);
    if (fe == 0) {
        const MRec ro = m.reco[k];
        lane_cells(box, ro, lane, d0, d1, v0, v1);
    } else {
        d0 = c0, d1 = c1, v0 = w0, v1 = w1;
    }
    const size_t N = box.nbox;
    float acc[10];
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = w0 * ba.u[c * N + c0] + w1 * ba.u[c * N + c1];
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[3 + c] = v0 * ba.s[c * N + d0] + v1 * ba.s[c * N + d1];
    acc[9] = v0 * ba.p[d0] + v1 * ba.p[d1];
#pragma unroll
    for (int c = 0; c < 10; ++c)
#pragma unroll
        for (int q = 16; q > 0; q >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], q);
    if (lane == 0) {
        // l = 0: h_k = U_k - I[u*](X_k); traction dS sigma(X_k) n_k and its moment
        const float dS = m.dS[k];
        for (int c = 0; c < 3; ++c) {
            const float h = m.U[c * nm + k] - acc[c];
            m.r0[c * nm + k] = h;
            if (!warm) {
                m.hl[c * nm + k] = h;
                m.rec[k].hdS[c] = h * dS;
            }
        }
        const float sxx = acc[3], syy = acc[4], szz = acc[5], sxy = acc[6], sxz = acc[7], syz = acc[8];
        const float nx = m.n[k], ny = m.n[nm + k], nz = m.n[2 * nm + k];
        const float dA = fe == 0 ? m.dSo[k] : dS;  // area of the surface the stress is taken on
        const float f0 = dA * (sxx * nx + sxy * ny + sxz * nz);
        const float f1 = dA * (sxy * nx + syy * ny + syz * nz);
        const float f2 = dA * (sxz * nx + syz * ny + szz * nz);
        const float off = fe == 0 ? F_OFFSET : 0.0f;
        const float r0 = m.arm[k] + off * nx, r1 = m.arm[nm + k] + off * ny, r2 = m.arm[2 * nm + k] + off * nz;
        m.ft[k] = f0;
        m.ft[nm + k] = f1;
        m.ft[2 * nm + k] = f2;
        m.ft[3 * nm + k] = r1 * f2 - r2 * f1;
        m.ft[4 * nm + k] = r2 * f0 - r0 * f2;
        m.ft[5 * nm + k] = r0 * f1 - r1 * f0;
        // the isotropic part -p I of sigma alone: the pressure force
        const float pdS = -dA * acc[9];
        m.ft[6 * nm + k] = pdS * nx;
        m.ft[7 * nm + k] = pdS * ny;
        m.ft[8 * nm + k] = pdS * nz;
    }
}


template <int NT>
__device__ __forceinline__ void interp0_block(const BoxGeom &box, int nm, const MarkerArrays &m, const BoxArrays &ba,
                                              const int *__restrict__ wlist, const int *__restrict__ wcount,
                                              int cap, DevState *st, int k, int warm) {
    constexpr int NW = NT / 32;
    constexpr int CU = 4;
    __shared__ int wc[CU][NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const MRec rk = m.rec[k];
    const int bx = rk.base & 1023, by = (rk.base >> 10) & 1023, bz = (rk.base >> 20) & 1023;
    if (warp == 0) interp_marker_warp(box, nm, m, ba, k, rk, lane, warm);
    // ---- row k of A -----------------------------------------------------------
    const int tile = (bx / TILE) + box.tx * ((by / TILE) + box.ty * (bz / TILE));
    const int cnt = wcount[tile];
    const int *list = wlist + (size_t)tile * cap;
    float *arow = m.aval + (size_t)k * ROWCAP;
    int *irow = m.aidx + (size_t)k * ROWCAP;
    int len = 0;
    // CU chunks of NT candidates per pass: their loads are issued together and
    // their hits are compacted chunk after chunk (list order, as one chunk at a time)
    for (int base = 0; base < cnt; base += CU * NT) {
        bool hit[CU];
        float a[CU];
        int j[CU];
#pragma unroll
        for (int u = 0; u < CU; ++u) {
            const int ii = base + u * NT + tid;
            j[u] = ii < cnt ? __ldg(list + ii) : -1;
        }
#pragma unroll
        for (int u = 0; u < CU; ++u) {
            hit[u] = false;
            a[u] = 0.0f;
            if (j[u] >= 0) {
                const MRec rj = m.rec[j[u]];
                const int dx = (rj.base & 1023) - bx, dy = ((rj.base >> 10) & 1023) - by,
                          dz = ((rj.base >> 20) & 1023) - bz;
                if (dx >= -3 && dx <= 3 && dy >= -3 && dy <= 3 && dz >= -3 && dz <= 3) {
                    a[u] = m.dS[j[u]] * overlap4(rk.wx, rj.wx, dx) * overlap4(rk.wy, rj.wy, dy) *
                           overlap4(rk.wz, rj.wz, dz);
                    hit[u] = true;
                }
            }
        }
        unsigned bal[CU];
#pragma unroll
        for (int u = 0; u < CU; ++u) {
            bal[u] = __ballot_sync(0xffffffffu, hit[u]);
            if (lane == 0) wc[u][warp] = __popc(bal[u]);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < CU; ++u) {
            int off = len, tot = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                if (w < warp) off += wc[u][w];
                tot += wc[u][w];
            }
            if (hit[u]) {
                const int pos = off + __popc(bal[u] & ((1u << lane) - 1u));
                if (pos < ROWCAP) {
                    arow[pos] = a[u];
                    irow[pos] = j[u];
                }
            }
            len += tot;
        }
        __syncthreads();
    }
    if (tid == 0) {
        m.alen[k] = len < ROWCAP ? len : ROWCAP;
        if (len > ROWCAP) atomicCAS(&st->status, 0, STAT_OVERFLOW);
    }
}

// 64 threads per marker: the blocks sit on the SMs beside the bulk
// collide+stream for the latency of their loads, so idle threads are costly.
constexpr int ROWS_MARKER_THREADS = 64;

__global__ void __launch_bounds__(ROWS_MARKER_THREADS) k_interp0_rows(BoxGeom box, int nm, MarkerArrays m,
                                                                      BoxArrays ba, const int *__restrict__ wlist,
                                                                      const int *__restrict__ wcount, int cap,
                                                                      DevState *st, int warm) {
    interp0_block<ROWS_MARKER_THREADS>(box, nm, m, ba, wlist, wcount, cap, st, blockIdx.x, warm);
}

// The same step l = 0 and rows of A with one block per TILE^3 tile of the
// support box, for batched launches (many markers, throughput-bound): the
// block finds the markers whose stencil base lies in the tile (from the
// tile's list 0, in marker order), interpolates each with one warp (the code
// above), and builds their rows from the tile's list 1 staged once in shared
// memory in chunks, one warp per marker and one candidate per lane with warp
// ordered compaction.  Entries and their order equal those of interp0_block.
constexpr int IT_MAXB = 256;   // markers based in one tile
constexpr int IT_STAGE = 256;  // candidates staged per chunk

__device__ __forceinline__ void interp0_tile_block(const BoxGeom &box, int nm, const MarkerArrays &m,
                                                   const BoxArrays &ba, const int *__restrict__ tile_list,
                                                   const int *__restrict__ tile_count, int cap, DevState *st,
                                                   int tile, int warm) {
    __shared__ int kb[IT_MAXB], klen[IT_MAXB];
    __shared__ int wc[ROWS_WARPS];
    __shared__ int nbased;
    __shared__ int sidx[IT_STAGE], sbase[IT_STAGE];
    // candidate weights per axis padded with three zeros on either side:
    // sp[a][3 + e][j] = w_a[e] of candidate j, so the overlap at base offset d
    // reads sp[a][i - d + 3] for i = 0..3 without branches; the padding adds
    // fmaf(w, 0, o) = o exactly (all weights are non-negative)
    __shared__ float sp[3][10][IT_STAGE];
    __shared__ float sdS[IT_STAGE];
    const int ntiles = box.tx * box.ty * box.tz;
    const int c0 = tile_count[tile];
    if (c0 == 0) return;  // no stencil overlaps the tile: no marker is based in it
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tile % box.tx, ty = (tile / box.tx) % box.ty, tz = tile / (box.tx * box.ty);
    const int *l0 = tile_list + (size_t)tile * cap;
    if (tid == 0) nbased = 0;
    __syncthreads();
    for (int base = 0; base < c0; base += ROWS_THREADS) {
        const int i = base + tid;
        bool hit = false;
        int k = 0;
        if (i < c0) {
            k = __ldg(l0 + i);
            const int pb = __ldg(m.base + k);
            hit = ((pb & 1023) / TILE == tx) && (((pb >> 10) & 1023) / TILE == ty) && (((pb >> 20) & 1023) / TILE == tz);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) wc[warp] = __popc(bal);
        __syncthreads();
        int off = nbased;
        for (int w = 0; w < warp; ++w) off += wc[w];
        if (hit) {
            const int pos = off + __popc(bal & ((1u << lane) - 1u));
            if (pos < IT_MAXB) kb[pos] = k;
        }
        __syncthreads();
        if (tid == 0) {
            int sum = 0;
            for (int w = 0; w < ROWS_WARPS; ++w) sum += wc[w];
            nbased += sum;
        }
        __syncthreads();
    }
    const int nb = nbased < IT_MAXB ? nbased : IT_MAXB;
    if (tid == 0 && nbased > IT_MAXB) atomicCAS(&st->status, 0, STAT_OVERFLOW);
    if (nb == 0) return;
    for (int q = warp; q < nb; q += ROWS_WARPS) {
        const int k = kb[q];
        const MRec rk = m.rec[k];
        interp_marker_warp(box, nm, m, ba, k, rk, lane, warm);
    }
    for (int q = tid; q < nb; q += ROWS_THREADS) klen[q] = 0;
    for (int q = tid; q < 3 * 6 * IT_STAGE; q += ROWS_THREADS) {
        const int a = q / (6 * IT_STAGE), r = (q / IT_STAGE) % 6, j = q % IT_STAGE;
        sp[a][r < 3 ? r : r + 4][j] = 0.0f;
    }
    const int c1 = tile_count[ntiles + tile];
    const int *l1 = tile_list + ((size_t)ntiles + tile) * cap;
    for (int base = 0; base < c1; base += IT_STAGE) {
        const int n = min(IT_STAGE, c1 - base);
        __syncthreads();  // the previous chunk is consumed (and klen is set)
        if (tid < n) {
            const int j = __ldg(l1 + base + tid);
            const MRec r = m.rec[j];
            sidx[tid] = j;
            sbase[tid] = r.base;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                sp[0][3 + e][tid] = r.wx[e];
                sp[1][3 + e][tid] = r.wy[e];
                sp[2][3 + e][tid] = r.wz[e];
            }
            sdS[tid] = m.dS[j];
        }
        __syncthreads();
        for (int q = warp; q < nb; q += ROWS_WARPS) {
            const int k = kb[q];
            const MRec rk = m.rec[k];
            const int bx = rk.base & 1023, by = (rk.base >> 10) & 1023, bz = (rk.base >> 20) & 1023;
            float *arow = m.aval + (size_t)k * ROWCAP;
            int *irow = m.aidx + (size_t)k * ROWCAP;
            int len = klen[q];
            for (int s0 = 0; s0 < n; s0 += 32) {
                const int jj = (s0 + lane < n) ? s0 + lane : 0;
                const int pb = sbase[jj];
                const int dx = (pb & 1023) - bx, dy = ((pb >> 10) & 1023) - by, dz = ((pb >> 20) & 1023) - bz;
                const bool hit = (s0 + lane < n) && dx >= -3 && dx <= 3 && dy >= -3 && dy <= 3 && dz >= -3 && dz <= 3;
                // the same fmaf sequence as overlap4, evaluated for every lane
                const int ox = 3 - min(max(dx, -3), 3), oy = 3 - min(max(dy, -3), 3), oz = 3 - min(max(dz, -3), 3);
                float fx = 0.0f, fy = 0.0f, fz = 0.0f;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    fx = fmaf(rk.wx[i], sp[0][i + ox][jj], fx);
                    fy = fmaf(rk.wy[i], sp[1][i + oy][jj], fy);
                    fz = fmaf(rk.wz[i], sp[2][i + oz][jj], fz);
                }
                const float a = sdS[jj] * fx * fy * fz;
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    const int pos = len + __popc(bal & ((1u << lane) - 1u));
                    if (pos < ROWCAP) {
                        arow[pos] = a;
                        irow[pos] = sidx[jj];
                    }
                }
                len += __popc(bal);
            }
            if (lane == 0) klen[q] = len;
        }
    }
    __syncthreads();
    for (int q = tid; q < nb; q += ROWS_THREADS) {
        const int len = klen[q];
        m.alen[kb[q]] = len < ROWCAP ? len : ROWCAP;
        if (len > ROWCAP) atomicCAS(&st->status, 0, STAT_OVERFLOW);
    }
}

__global__ void __launch_bounds__(ROWS_THREADS) k_interp0_tiles(BoxGeom box, int nm, MarkerArrays m, BoxArrays ba,
                                                                 const int *__restrict__ tile_list,
                                                                 const int *__restrict__ tile_count, int cap,
                                                                 DevState *st, int warm) {
    interp0_tile_block(box, nm, m, ba, tile_list, tile_count, cap, st, blockIdx.x, warm);
}

// One cycle of steps l = 1..4 (Sec. 2.2) in matrix form:
//   h_out_k = h_in_k + U_k - I[u* + S h_in](X_k) = h_in_k + r0_k - sum_j A_kj h_in_j.
// One warp per marker, entries of the row in order per lane, xor-shuffle sum.
// The last cycle also stores h dS for the spreading of h_imm.
// adaptive (predictor modes): cycle `cyc` (0-based) is skipped -- h_out = h_in
// -- once the slip max_k |U_k - I[u* + S h_in](X_k)| = max |r0 - A h_in| seen
// by cycle cyc - 1 is below eps; each executed cycle records its slip (an
// atomic maximum of non-negative float bits: exact, order-independent).
// h_final: also receives the last cycle's h when that is not h_out.
__device__ __forceinline__ void cycle_block(int nm, const MarkerArrays &m, const float *__restrict__ h_in,
                                            float *__restrict__ h_out, float *__restrict__ h_final, int last,
                                            int blk, DevState *st, int cyc, int adaptive, float eps) {
    __shared__ float smax[INTERP_WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blk * INTERP_WARPS + warp;
    const bool skip = adaptive && cyc > 0 && __uint_as_float(st->pr.slip[cyc - 1]) < eps;
    float res_max = 0.0f;
    if (k < nm) {
        const float dS = m.dS[k];
        if (skip) {
            if (lane == 0)
                for (int c = 0; c < 3; ++c) {
                    const float h = h_in[c * nm + k];
                    h_out[c * nm + k] = h;
                    if (last) m.rec[k].hdS[c] = h * dS;
                    if (last && h_final) h_final[c * nm + k] = h;
                }
        } else {
            const int len = m.alen[k];
            const float *arow = m.aval + (size_t)k * ROWCAP;
            const int *irow = m.aidx + (size_t)k * ROWCAP;
            float ax = 0.0f, ay = 0.0f, az = 0.0f;
            // lane l adds entries l, l + 32, l + 64, ... in that order; the loads of
            // four of them are issued together (two memory round trips per 128
            // entries instead of two per 32), the first four beside the row length
            constexpr int U = 4;
            for (int e0 = 0; e0 == 0 || e0 < len; e0 += 32 * U) {
                float a[U], hx[U], hy[U], hz[U];
                int j[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + 32 * u + lane;
                    a[u] = e < ROWCAP ? arow[e] : 0.0f;
                    const int jj = e < ROWCAP ? irow[e] : k;
                    j[u] = (unsigned)jj < (unsigned)nm ? jj : k;  // entries past the row: any valid index
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    hx[u] = h_in[j[u]];
                    hy[u] = h_in[nm + j[u]];
                    hz[u] = h_in[2 * nm + j[u]];
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (e0 + 32 * u + lane < len) {
                        ax = fmaf(a[u], hx[u], ax);
                        ay = fmaf(a[u], hy[u], ay);
                        az = fmaf(a[u], hz[u], az);
                    }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
                az += __shfl_xor_sync(0xffffffffu, az, o);
            }
            if (lane == 0) {
                const float acc[3] = {ax, ay, az};
                for (int c = 0; c < 3; ++c) {
                    const float res = m.r0[c * nm + k] - acc[c];
                    const float h = h_in[c * nm + k] + res;
                    h_out[c * nm + k] = h;
                    if (last) m.rec[k].hdS[c] = h * dS;
                    if (last && h_final) h_final[c * nm + k] = h;
                    res_max = fmaxf(res_max, fabsf(res));
                }
            }
        }
    }
    if (skip) return;  // uniform over the block
    if (lane == 0) smax[warp] = res_max;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = smax[0];
        for (int w = 1; w < INTERP_WARPS; ++w) b = fmaxf(b, smax[w]);
        if (cyc < 8) atomicMax(&st->pr.slip[cyc], __float_as_uint(b));
        if (blk == 0) st->pr.cycles += 1;
    }
}

__global__ void __launch_bounds__(32 * INTERP_WARPS) k_cycle(int nm, MarkerArrays m, const float *__restrict__ h_in,
                                                             float *__restrict__ h_out, float *__restrict__ h_final,
                                                             int last, DevState *st, int cyc, int adaptive,
                                                             float eps) {
    cycle_block(nm, m, h_in, h_out, h_final, last, blockIdx.x, st, cyc, adaptive, eps);
}

// F = sum_k dS sigma.n, T = sum_k arm x (dS sigma.n) and the pressure part
// Fp = sum_k -dS p n in FP64: warp c (of 9) sums component c, lane l the
// markers l, l+32, ... in order, then an xor tree.
// Then, in thread 0: the relative error of the prediction made for this time
// level (predictor modes: a large one switches the next prediction to the
// linear one), the force/torque history, and the trajectory record of time
// level st->s[slot] (when a log is attached).
__device__ __forceinline__ void reduce_block(int nm, const float *__restrict__ ft, DevState *st, int slot,
                                             int predictor, int opts, double theta, double *__restrict__ log,
                                             long long log_cap) {
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // eight independent partial sums per lane, so that eight loads are in
    // flight at a time; combined in a fixed order (reproducible)
    double a8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const float *fc = ft + (size_t)c * nm;
    int k = lane;
    for (; k + 7 * 32 < nm; k += 8 * 32) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(fc + k + u * 32);
#pragma unroll
        for (int u = 0; u < 8; ++u) a8[u] += (double)v[u];
    }
#pragma unroll
    for (int u = 0; u < 7; ++u)
        if (k + u * 32 < nm) a8[u] += (double)__ldg(fc + k + u * 32);
    double a = ((a8[0] + a8[1]) + (a8[2] + a8[3])) + ((a8[4] + a8[5]) + (a8[6] + a8[7]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) {
        if (c < 3) st->F[c] = a; else if (c < 6) st->T[c - 3] = a; else st->Fp[c - 6] = a;
        if (!isfinite(a)) atomicCAS(&st->status, 0, STAT_DIVERGED);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    Predictor &P = st->pr;
    double resid = -1.0, resid_net = -1.0, made = -1.0, fh[6] = {0, 0, 0, 0, 0, 0};
    auto rel_err = [&](const double *Fp) {
        double num = 0.0, den = 0.0;
        for (int q = 0; q < 3; ++q) {
            num += (st->F[q] - Fp[q]) * (st->F[q] - Fp[q]);
            den += st->F[q] * st->F[q];
        }
        return den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
    };
    if (predictor != 0 && P.predicted) {
        made = P.by_net ? 1.0 : 0.0;
        for (int q = 0; q < 3; ++q) {
            fh[q] = P.Fhat[q];
            fh[3 + q] = P.That[q];
        }
        resid = rel_err(P.Fhat);
        P.resid = resid;
        P.predicted = 0;
    }
    if (predictor != 0 && P.net_ok) {  // the network's own accuracy decides the fallback
        resid_net = rel_err(P.Fnet);
        P.resid_net = resid_net;
        if (opts & PRED_REL) {
            // relative rule: running means of the network's error and of linear
            // extrapolation's error on the same time levels; the network is used
            // while its mean is at most theta times the linear one
            double Flin[3];
            for (int q = 0; q < 3; ++q) Flin[q] = 2.0 * P.Fh[0][q] - P.Fh[1][q];
            const double rl = rel_err(Flin);
            const bool first = P.ema_lin == 0.0 && P.ema_net == 0.0;
            P.ema_net = first ? resid_net : P.ema_net + 0.125 * (resid_net - P.ema_net);
            P.ema_lin = first ? rl : P.ema_lin + 0.125 * (rl - P.ema_lin);
            P.fallback = !(P.ema_net <= theta * P.ema_lin);
        } else {
            P.fallback = !(resid_net <= theta);
        }
        P.net_ok = 0;
    }
    for (int h = 3; h > 0; --h)
        for (int q = 0; q < 3; ++q) {
            P.Fh[h][q] = P.Fh[h - 1][q];
            P.Th[h][q] = P.Th[h - 1][q];
        }
    for (int q = 0; q < 3; ++q) {
        P.Fh[0][q] = st->F[q];
        P.Th[0][q] = st->T[q];
    }
    P.hist_n = P.hist_n < 4 ? P.hist_n + 1 : 4;
    if (log && log_cap > 0) {
        const BodySlot &S = st->s[slot];
        double *r = log + (size_t)(P.logged % log_cap) * LOG_REC;
        for (int q = 0; q < 9; ++q) r[q] = S.d[q];
        for (int q = 0; q < 3; ++q) {
            r[9 + q] = S.v[q];
            r[12 + q] = S.w[q];
            r[15 + q] = st->F[q];
            r[18 + q] = st->T[q];
        }
        r[21] = (double)S.step;
        r[22] = resid;
        for (int q = 0; q < 6; ++q) r[23 + q] = fh[q];
        r[29] = made;
        r[30] = resid_net;
        r[31] = 0.0;
    }
    P.logged += 1;
}

__global__ void __launch_bounds__(288) k_reduce_ft(int nm, const float *__restrict__ ft, DevState *st, int slot,
                                                   int predictor, int opts, double theta,
                                                   double *__restrict__ log, long long log_cap) {
    reduce_block(nm, ft, st, slot, predictor, opts, theta, log, log_cap);
}

constexpr int SPREAD_SLICES = 8;                               // candidate slices per tile
constexpr int SPREAD_THREADS = TILE * TILE * TILE * SPREAD_SLICES;  // 64 cells x 8 slices
constexpr int SPREAD_STAGE = 256;

// h_imm(x) = S[h](x) = sum_k W(x - X_k) h_k dS_k on the support box.  One block
// per 4^3 tile: the tile's candidate records are staged in shared memory as
// structure of arrays; thread (cell c, slice q) sums slice q of each staged
// chunk for cell c; the 8 slice sums are added in slice order (reproducible).
__device__ __forceinline__ void spread_block(const BoxGeom &box, const MRec *__restrict__ rec, const BoxArrays &ba,
                                             const int *__restrict__ tile_list, const int *__restrict__ tile_count,
                                             int cap, int tile) {
    constexpr int TC = TILE * TILE * TILE;
    __shared__ int sbase[SPREAD_STAGE];
    __shared__ float sw[12][SPREAD_STAGE];
    __shared__ float sh[3][SPREAD_STAGE];
    __shared__ float part[SPREAD_SLICES][3][TC];
    const int cnt = tile_count[tile];
    const int tx = tile % box.tx, ty = (tile / box.tx) % box.ty, tz = tile / (box.tx * box.ty);
    const int tid = threadIdx.x, c = tid % TC, q = tid / TC;
    const int cx = TILE * tx + c % TILE, cy = TILE * ty + (c / TILE) % TILE, cz = TILE * tz + c / (TILE * TILE);
    const int *list = tile_list + (size_t)tile * cap;
    float ax = 0.0f, ay = 0.0f, az = 0.0f;
    for (int base = 0; base < cnt; base += SPREAD_STAGE) {
        const int n = min(SPREAD_STAGE, cnt - base);
        if (tid < n) {
            const MRec r = rec[__ldg(list + base + tid)];
            sbase[tid] = r.base;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                sw[e][tid] = r.wx[e];
                sw[4 + e][tid] = r.wy[e];
                sw[8 + e][tid] = r.wz[e];
            }
            sh[0][tid] = r.hdS[0];
            sh[1][tid] = r.hdS[1];
            sh[2][tid] = r.hdS[2];
        }
        __syncthreads();
        const int j0 = (n * q) / SPREAD_SLICES, j1 = (n * (q + 1)) / SPREAD_SLICES;
        for (int jj = j0; jj < j1; ++jj) {
            const int pb = sbase[jj];
            const int dx = cx - (pb & 1023), dy = cy - ((pb >> 10) & 1023), dz = cz - ((pb >> 20) & 1023);
            if ((unsigned)dx < 4u && (unsigned)dy < 4u && (unsigned)dz < 4u) {
                const float wv = sw[dx][jj] * sw[4 + dy][jj] * sw[8 + dz][jj];
                ax = fmaf(wv, sh[0][jj], ax);
                ay = fmaf(wv, sh[1][jj], ay);
                az = fmaf(wv, sh[2][jj], az);
            }
        }
        __syncthreads();
    }
    part[q][0][c] = ax;
    part[q][1][c] = ay;
    part[q][2][c] = az;
    __syncthreads();
    if (tid < TC) {
        float hx = 0.0f, hy = 0.0f, hz = 0.0f;
#pragma unroll
        for (int w = 0; w < SPREAD_SLICES; ++w) {  // fixed slice order: reproducible
            hx += part[w][0][tid];
            hy += part[w][1][tid];
            hz += part[w][2][tid];
        }
        if (cx < box.Bx && cy < box.By && cz < box.Bz) {
            const size_t b = ((size_t)cz * box.By + cy) * box.Bx + cx;
            ba.h[b] = hx;
            ba.h[box.nbox + b] = hy;
            ba.h[2 * box.nbox + b] = hz;
        }
    }
}

__global__ void __launch_bounds__(SPREAD_THREADS) k_spread(BoxGeom box, const MRec *__restrict__ rec, BoxArrays ba,
                                                           const int *__restrict__ tile_list,
                                                           const int *__restrict__ tile_count, int cap) {
    spread_block(box, rec, ba, tile_list, tile_count, cap, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Batched forms: one launch per phase over all runs of a batch, block b of
// the launch serving block b - prefix[r] of run r (prefix[r] <= b <
// prefix[r + 1]), with the same block code as the single-run kernels.

__global__ void __launch_bounds__(PM_THREADS) k_batch_particle_markers(const RunDesc *__restrict__ runs,
                                                                        const int *__restrict__ prefix, int nruns,
                                                                        int p) {
    int lb;
    const RunDesc &R = runs[block_run(prefix, nruns, lb)];
    pm_block(R.g, R.bc, R.box, R.st, p, 1, R.m, lb);
}

__global__ void __launch_bounds__(ROWS_THREADS) k_batch_interp0_tiles(const RunDesc *__restrict__ runs,
                                                                      const int *__restrict__ prefix, int nruns,
                                                                      int warm) {
    int lb;
    const RunDesc &R = runs[block_run(prefix, nruns, lb)];
    interp0_tile_block(R.box, R.nm, R.m, R.ba, R.tile_list, R.tile_count, R.cap, R.st, lb, warm);
}

__device__ __forceinline__ float *hsel(const MarkerArrays &m, int sel) {
    return sel == HSEL_R0 ? m.r0 : (sel == HSEL_HL ? m.hl : m.hb);
}

__global__ void __launch_bounds__(32 * INTERP_WARPS) k_batch_cycle(const RunDesc *__restrict__ runs,
                                                                   const int *__restrict__ prefix, int nruns,
                                                                   int sel_in, int sel_out, int sel_final, int last,
                                                                   int cyc, int adaptive) {
    int lb;
    const RunDesc &R = runs[block_run(prefix, nruns, lb)];
    cycle_block(R.nm, R.m, hsel(R.m, sel_in), hsel(R.m, sel_out), sel_final >= 0 ? hsel(R.m, sel_final) : nullptr,
                last, lb, R.st, cyc, adaptive, R.bc.slip_eps);
}

__global__ void __launch_bounds__(288) k_batch_reduce_ft(const RunDesc *__restrict__ runs, int slot) {
    const RunDesc &R = runs[blockIdx.x];
    reduce_block(R.nm, R.m.ft, R.st, slot, R.bc.predictor, R.bc.pred_opts, R.bc.resid_theta, R.bc.log, R.bc.log_cap);
}

__global__ void __launch_bounds__(SPREAD_THREADS) k_batch_spread(const RunDesc *__restrict__ runs,
                                                                 const int *__restrict__ prefix, int nruns) {
    int lb;
    const RunDesc &R = runs[block_run(prefix, nruns, lb)];
    spread_block(R.box, R.m.rec, R.ba, R.tile_list, R.tile_count, R.cap, lb);
}

// ---------------------------------------------------------------------------
cudaError_t launch_particle_markers(const Geom &g, const BodyConst &bc, const BoxGeom &box, DevState *st, int slot,
                                    int advance, MarkerArrays m, cudaStream_t s) {
    k_particle_markers<<<(bc.nm + PM_THREADS - 1) / PM_THREADS, PM_THREADS, 0, s>>>(g, bc, box, st, slot, advance, m);
    return cudaGetLastError();
}

cudaError_t launch_interp0(const BoxGeom &box, int nm, MarkerArrays m, BoxArrays ba, const int *tile_list,
                           const int *tile_count, int cap, DevState *st, int warm, cudaStream_t s, bool by_tile) {
    const int ntiles = box.tx * box.ty * box.tz;  // list 1 (rows of A) follows list 0
    if (by_tile)
        k_interp0_tiles<<<ntiles, ROWS_THREADS, 0, s>>>(box, nm, m, ba, tile_list, tile_count, cap, st, warm);
    else
        k_interp0_rows<<<nm, ROWS_MARKER_THREADS, 0, s>>>(box, nm, m, ba, tile_list + (size_t)ntiles * cap,
                                                   tile_count + ntiles, cap, st, warm);
    return cudaGetLastError();
}

cudaError_t launch_cycle(int nm, MarkerArrays m, const float *h_in, float *h_out, float *h_final, int last,
                         DevState *st, int cyc, int adaptive, float eps, cudaStream_t s) {
    k_cycle<<<(nm + INTERP_WARPS - 1) / INTERP_WARPS, 32 * INTERP_WARPS, 0, s>>>(nm, m, h_in, h_out, h_final, last,
                                                                                 st, cyc, adaptive, eps);
    return cudaGetLastError();
}

cudaError_t launch_reduce_ft(int nm, MarkerArrays m, DevState *st, int slot, const BodyConst &bc, cudaStream_t s) {
    k_reduce_ft<<<1, 288, 0, s>>>(nm, m.ft, st, slot, bc.predictor, bc.pred_opts, bc.resid_theta, bc.log, bc.log_cap);
    return cudaGetLastError();
}

cudaError_t launch_spread(const BoxGeom &box, int nm, MarkerArrays m, BoxArrays ba, const int *tile_list,
                          const int *tile_count, int cap, cudaStream_t s) {
    (void)nm;
    k_spread<<<box.tx * box.ty * box.tz, SPREAD_THREADS, 0, s>>>(box, m.rec, ba, tile_list, tile_count, cap);
    return cudaGetLastError();
}

int blocks_particle_markers(const RunDesc &r) { return (r.nm + PM_THREADS - 1) / PM_THREADS; }
int blocks_interp0(const RunDesc &r) { return r.box.tx * r.box.ty * r.box.tz; }
int blocks_cycle(const RunDesc &r) { return (r.nm + INTERP_WARPS - 1) / INTERP_WARPS; }
int blocks_spread(const RunDesc &r) { return r.box.tx * r.box.ty * r.box.tz; }

cudaError_t launch_batch_particle_markers(const RunDesc *runs, const int *prefix, int nruns, int p, int nblocks,
                                          cudaStream_t s) {
    k_batch_particle_markers<<<nblocks, PM_THREADS, 0, s>>>(runs, prefix, nruns, p);
    return cudaGetLastError();
}

cudaError_t launch_batch_interp0(const RunDesc *runs, const int *prefix, int nruns, int nblocks, int warm,
                                 cudaStream_t s) {
    k_batch_interp0_tiles<<<nblocks, ROWS_THREADS, 0, s>>>(runs, prefix, nruns, warm);
    return cudaGetLastError();
}

cudaError_t launch_batch_cycle(const RunDesc *runs, const int *prefix, int nruns, int nblocks, int sel_in,
                               int sel_out, int sel_final, int last, int cyc, int adaptive, cudaStream_t s) {
    k_batch_cycle<<<nblocks, 32 * INTERP_WARPS, 0, s>>>(runs, prefix, nruns, sel_in, sel_out, sel_final, last, cyc,
                                                        adaptive);
    return cudaGetLastError();
}

cudaError_t launch_batch_reduce_ft(const RunDesc *runs, int nruns, int slot, cudaStream_t s) {
    k_batch_reduce_ft<<<nruns, 288, 0, s>>>(runs, slot);
    return cudaGetLastError();
}

cudaError_t launch_batch_spread(const RunDesc *runs, const int *prefix, int nruns, int nblocks, cudaStream_t s) {
    k_batch_spread<<<nblocks, SPREAD_THREADS, 0, s>>>(runs, prefix, nruns);
    return cudaGetLastError();
}

}  // namespace turret
