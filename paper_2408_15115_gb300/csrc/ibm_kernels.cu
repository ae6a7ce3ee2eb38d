// ibm_kernels.cu -- rigid-body update, marker kinematics and the
// immersed-boundary transfers of the Palabos Turret step (arXiv 2408.15115).
//
//   k_particle : FP64 leap-frog 6DOF with the orientation predictor-corrector
//                (Sec. 2.3), then the vertical window slide; one thread.
//   k_markers  : X_k = C_m + M^T Xb_k, n_k = M^T nb_k, U_k = v + w x (X_k - C_m)
//                (Sec. 2.3 end), the 4x4x4 Peskin stencil base of each marker in
//                support-box coordinates and its 12 one-dimensional weights
//                (Sec. 2.2), one thread per marker.
//   k_bin      : for every 8^3 tile of the support box, the markers whose
//                stencil overlaps it, in marker order (ordered compaction).
//   k_interp   : I[u](X_k) = sum_x u(x) W(x - X_k), one warp per marker, two
//                stencil cells per lane, xor-shuffle reduction (deterministic);
//                mode 0 also interpolates sigma and forms dS sigma.n and the
//                torque arm product for the surface force (Sec. 2.2 end).
//   k_spread   : S[h](x) = sum_k h_k W(x - X_k) dS_k as a gather: one block
//                per tile, each cell sums its tile's candidate list in marker
//                order -- no atomics, bitwise reproducible.
//   k_reduce_ft: F = sum_k f_k, T = sum_k t_k in FP64, fixed-order block
//                partials and a last-block final sum.
#include <math.h>

#include "turret_internal.cuh"

namespace turret {

__device__ __forceinline__ void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__global__ void k_particle(Geom g, BodyConst bc, DevState *__restrict__ stp) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DevState s = *stp;
    for (int a = 0; a < 3; ++a) {
        s.v[a] += bc.g_eff[a] + s.F[a] / bc.mass;  // a(t) = g_eff + F(t)/(kappa V)
        s.r[a] += s.v[a];
    }
    double src[3];
    for (int a = 0; a < 3; ++a) {
        if (bc.rot_form == 1) {
            src[a] = s.T[a];
        } else {
            s.L[a] += s.T[a];
            src[a] = s.L[a];
        }
    }
    double sb[3], wb[3], wl[3];
    for (int i = 0; i < 3; ++i) sb[i] = s.d[3 * i] * src[0] + s.d[3 * i + 1] * src[1] + s.d[3 * i + 2] * src[2];
    for (int i = 0; i < 3; ++i)
        wb[i] = (bc.Jinv_b[3 * i] * sb[0] + bc.Jinv_b[3 * i + 1] * sb[1] + bc.Jinv_b[3 * i + 2] * sb[2]) / bc.mass;
    for (int a = 0; a < 3; ++a) wl[a] = s.d[a] * wb[0] + s.d[3 + a] * wb[1] + s.d[6 + a] * wb[2];
    for (int a = 0; a < 3; ++a) s.w[a] = (bc.rot_form == 1) ? s.w[a] + wl[a] : wl[a];
    double dn[9];
    for (int i = 0; i < 3; ++i) {
        double c1[3], pred[3], mid[3], c2[3];
        cross3(s.w, s.d + 3 * i, c1);
        for (int a = 0; a < 3; ++a) pred[a] = s.d[3 * i + a] + c1[a];
        for (int a = 0; a < 3; ++a) mid[a] = 0.5 * (s.d[3 * i + a] + pred[a]);
        cross3(s.w, mid, c2);
        for (int a = 0; a < 3; ++a) dn[3 * i + a] = s.d[3 * i + a] + c2[a];
    }
    for (int k = 0; k < 9; ++k) s.d[k] = dn[k];
    if (bc.renorm) {
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < i; ++j) {
                double pj = 0.0;
                for (int a = 0; a < 3; ++a) pj += s.d[3 * i + a] * s.d[3 * j + a];
                for (int a = 0; a < 3; ++a) s.d[3 * i + a] -= pj * s.d[3 * j + a];
            }
            const double l = sqrt(s.d[3 * i] * s.d[3 * i] + s.d[3 * i + 1] * s.d[3 * i + 1] + s.d[3 * i + 2] * s.d[3 * i + 2]);
            for (int a = 0; a < 3; ++a) s.d[3 * i + a] /= l;
        }
    }
    // vertical slide of the ring window: one plane per step at most
    s.reseed_plane = -1;
    if (bc.slide) {
        const double dz = (s.r[2] - (double)s.origin[2]) - bc.anchor_z;
        if (dz <= -1.0) {
            s.origin[2] -= 1;
            s.ring = (s.ring == 0) ? g.nz - 1 : s.ring - 1;
            s.reseed_plane = s.ring;  // new logical bottom plane
        } else if (dz >= 1.0) {
            s.origin[2] += 1;
            s.ring = (s.ring + 1 == g.nz) ? 0 : s.ring + 1;
            s.reseed_plane = (s.ring + g.nz - 1) % g.nz;  // new logical top plane
        }
    }
    for (int a = 0; a < 3; ++a) {
        const double C = s.r[a] - (double)s.origin[a];
        const double fl = floor(C);
        s.Ci[a] = (int)fl;
        s.Cf[a] = C - fl;
        s.box_lo[a] = s.Ci[a] - bc.rc - 2;
    }
    s.step += 1;
    *stp = s;
}

// Peskin 4-point kernel (Sec. 2.2) on the two branches, |r| given.
__device__ __forceinline__ float peskin_in(float a) { return 0.125f * (3.0f - 2.0f * a + sqrtf(1.0f + 4.0f * a - 4.0f * a * a)); }
__device__ __forceinline__ float peskin_out(float a) {
    return 0.125f * (5.0f - 2.0f * a - sqrtf(fmaxf(0.0f, -7.0f + 12.0f * a - 4.0f * a * a)));
}

__global__ void k_markers(Geom g, BodyConst bc, BoxGeom box, DevState *st, MarkerArrays m) {
    const DevState *st_c = st;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= bc.nm) return;
    const int nm = bc.nm;
    float d[9], v[3], w[3], cf[3];
    int ci[3], lo[3];
#pragma unroll
    for (int a = 0; a < 9; ++a) d[a] = (float)st_c->d[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v[a] = (float)st_c->v[a];
        w[a] = (float)st_c->w[a];
        cf[a] = (float)st_c->Cf[a];
        ci[a] = st_c->Ci[a];
        lo[a] = st_c->box_lo[a];
    }
    const float xb[3] = {m.Xb[k], m.Xb[nm + k], m.Xb[2 * nm + k]};
    const float nbv[3] = {m.nb[k], m.nb[nm + k], m.nb[2 * nm + k]};
    float arm[3], nn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        arm[a] = d[a] * xb[0] + d[3 + a] * xb[1] + d[6 + a] * xb[2];
        nn[a] = d[a] * nbv[0] + d[3 + a] * nbv[1] + d[6 + a] * nbv[2];
    }
    const float U[3] = {v[0] + (w[1] * arm[2] - w[2] * arm[1]), v[1] + (w[2] * arm[0] - w[0] * arm[2]),
                        v[2] + (w[0] * arm[1] - w[1] * arm[0])};
    const int n[3] = {g.nx, g.ny, g.nz};
    const bool per[3] = {g.bc_x == BC_PERIODIC, g.bc_y == BC_PERIODIC, g.bc_bottom == BC_PERIODIC};
    const int B[3] = {box.Bx, box.By, box.Bz};
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xr = cf[a] + arm[a];  // marker position relative to Ci
        const float fl = floorf(xr);
        const float t = xr - fl;          // in [0, 1)
        int base_rel = (int)fl - 1;       // stencil cells base_rel .. base_rel + 3
        int bbv = ci[a] + base_rel - lo[a];
        float w4[4] = {peskin_out(1.0f + t), peskin_in(t), peskin_in(1.0f - t), peskin_out(2.0f - t)};
        // a non-finite or out-of-box position must never index memory: park the
        // stencil at the box origin with zero weights and latch the status
        if (!isfinite(xr) || bbv < 0 || bbv > B[a] - 4) {
            bbv = 0;
            base_rel = lo[a] - ci[a];
            w4[0] = w4[1] = w4[2] = w4[3] = 0.0f;
            bad = true;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) m.wgt[(4 * a + q) * nm + k] = w4[q];
        m.bb[a * nm + k] = bbv;
        const int abs_base = ci[a] + base_rel;
        if (!per[a] && (abs_base < 0 || abs_base + 3 > n[a] - 1)) bad = true;
        m.U[a * nm + k] = U[a];
        m.n[a * nm + k] = nn[a];
        m.arm[a * nm + k] = arm[a];
    }
    if (bad) atomicCAS(&st->status, 0, STAT_DOMAIN);  // the first latched error wins
}

__global__ void __launch_bounds__(256) k_bin(BoxGeom box, int nm, const int *__restrict__ bb,
                                             int *__restrict__ tile_list, int *__restrict__ tile_count, int cap) {
    const int tile = blockIdx.x;
    const int tx = tile % box.tx, ty = (tile / box.tx) % box.ty, tz = tile / (box.tx * box.ty);
    const int t0[3] = {8 * tx, 8 * ty, 8 * tz};
    __shared__ int wcount[8];
    __shared__ int total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) total = 0;
    __syncthreads();
    for (int chunk = 0; chunk < nm; chunk += 256) {
        const int k = chunk + tid;
        bool hit = false;
        if (k < nm) {
            hit = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int b = bb[a * nm + k];
                hit = hit && (b <= t0[a] + 7) && (b + 3 >= t0[a]);
            }
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
    if (tid == 0) tile_count[tile] = total < cap ? total : cap;
}

__global__ void __launch_bounds__(128) k_interp(BoxGeom box, int nm, MarkerArrays m, BoxArrays ba, int mode) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= nm) return;
    const int i = lane & 3, j = (lane >> 2) & 3, kz = lane >> 4;
    const int bx = m.bb[k], by = m.bb[nm + k], bz = m.bb[2 * nm + k];
    const float wxy = m.wgt[i * nm + k] * m.wgt[(4 + j) * nm + k];
    const float w0 = wxy * m.wgt[(8 + kz) * nm + k];
    const float w1 = wxy * m.wgt[(10 + kz) * nm + k];
    const size_t c0 = ((size_t)(bz + kz) * box.By + (by + j)) * box.Bx + (bx + i);
    const size_t c1 = c0 + 2 * (size_t)box.By * box.Bx;
    const size_t N = box.nbox;
    float acc[9];
    const int nv = (mode == 0) ? 9 : 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float a0 = ba.u[c * N + c0], a1 = ba.u[c * N + c1];
        if (mode != 0) {
            a0 += ba.h[c * N + c0];
            a1 += ba.h[c * N + c1];
        }
        acc[c] = w0 * a0 + w1 * a1;
    }
    if (mode == 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[3 + c] = w0 * ba.s[c * N + c0] + w1 * ba.s[c * N + c1];
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        if (c >= nv) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    }
    if (lane != 0) return;
    if (mode == 0) {
        // l = 0: h_k = U_k - I[u*](X_k); surface traction dS sigma(X_k) n_k
        for (int c = 0; c < 3; ++c) m.hl[c * nm + k] = m.U[c * nm + k] - acc[c];
        const float sxx = acc[3], syy = acc[4], szz = acc[5], sxy = acc[6], sxz = acc[7], syz = acc[8];
        const float nx = m.n[k], ny = m.n[nm + k], nz = m.n[2 * nm + k], dS = m.dS[k];
        const float f[3] = {dS * (sxx * nx + sxy * ny + sxz * nz), dS * (sxy * nx + syy * ny + syz * nz),
                            dS * (sxz * nx + syz * ny + szz * nz)};
        const float r[3] = {m.arm[k], m.arm[nm + k], m.arm[2 * nm + k]};
        m.ft[k] = f[0];
        m.ft[nm + k] = f[1];
        m.ft[2 * nm + k] = f[2];
        m.ft[3 * nm + k] = r[1] * f[2] - r[2] * f[1];
        m.ft[4 * nm + k] = r[2] * f[0] - r[0] * f[2];
        m.ft[5 * nm + k] = r[0] * f[1] - r[1] * f[0];
    } else {
        // l = 4: h_k <- h_k + U_k - I[u* + S h](X_k)
        for (int c = 0; c < 3; ++c) m.hl[c * nm + k] += m.U[c * nm + k] - acc[c];
    }
}

__global__ void __launch_bounds__(256) k_reduce_ft(int nm, const float *__restrict__ ft, double *partials,
                                                   DevState *st) {
    __shared__ double sh[6][256];
    __shared__ bool last;
    const int tid = threadIdx.x, b = blockIdx.x;
    const int chunk = (nm + REDUCE_BLOCKS - 1) / REDUCE_BLOCKS;
    const int k0 = b * chunk, k1 = min(nm, k0 + chunk);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int k = k0 + tid; k < k1; k += 256)
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += (double)ft[c * nm + k];
#pragma unroll
    for (int c = 0; c < 6; ++c) sh[c][tid] = acc[c];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s)
#pragma unroll
            for (int c = 0; c < 6; ++c) sh[c][tid] += sh[c][tid + s];
        __syncthreads();
    }
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) partials[6 * b + c] = sh[c][0];
        __threadfence();
        const unsigned ticket = atomicAdd(&st->counter, 1u);
        last = (ticket == REDUCE_BLOCKS - 1);
    }
    __syncthreads();
    if (!last || tid != 0) return;
    __threadfence();
    double tot[6] = {0, 0, 0, 0, 0, 0};
    for (int bb = 0; bb < REDUCE_BLOCKS; ++bb)
#pragma unroll
        for (int c = 0; c < 6; ++c) tot[c] += __ldcg(partials + 6 * bb + c);
    bool finite = true;
    for (int c = 0; c < 3; ++c) {
        st->F[c] = tot[c];
        st->T[c] = tot[3 + c];
        finite = finite && isfinite(tot[c]) && isfinite(tot[3 + c]);
    }
    if (!finite) atomicCAS(&st->status, 0, STAT_DIVERGED);
    st->counter = 0;
}

__global__ void __launch_bounds__(512) k_spread(BoxGeom box, int nm, MarkerArrays m, BoxArrays ba,
                                                const int *__restrict__ tile_list, const int *__restrict__ tile_count,
                                                int cap) {
    constexpr int CH = 256;
    __shared__ int sb[3][CH];
    __shared__ float sw[12][CH];
    __shared__ float sh[3][CH];
    const int tile = blockIdx.x;
    const int tx = tile % box.tx, ty = (tile / box.tx) % box.ty, tz = tile / (box.tx * box.ty);
    const int tid = threadIdx.x;
    const int cx = 8 * tx + (tid & 7), cy = 8 * ty + ((tid >> 3) & 7), cz = 8 * tz + (tid >> 6);
    const int cnt = tile_count[tile];
    float ax = 0.0f, ay = 0.0f, az = 0.0f;
    for (int base = 0; base < cnt; base += CH) {
        if (tid < CH && base + tid < cnt) {
            const int k = tile_list[(size_t)tile * cap + base + tid];
#pragma unroll
            for (int a = 0; a < 3; ++a) sb[a][tid] = m.bb[a * nm + k];
#pragma unroll
            for (int q = 0; q < 12; ++q) sw[q][tid] = m.wgt[q * nm + k];
            const float dS = m.dS[k];
#pragma unroll
            for (int a = 0; a < 3; ++a) sh[a][tid] = m.hl[a * nm + k] * dS;
        }
        __syncthreads();
        const int nloc = min(CH, cnt - base);
        for (int jj = 0; jj < nloc; ++jj) {
            const int dx = cx - sb[0][jj], dy = cy - sb[1][jj], dz = cz - sb[2][jj];
            if ((unsigned)dx < 4u && (unsigned)dy < 4u && (unsigned)dz < 4u) {
                const float wv = sw[dx][jj] * sw[4 + dy][jj] * sw[8 + dz][jj];
                ax += wv * sh[0][jj];
                ay += wv * sh[1][jj];
                az += wv * sh[2][jj];
            }
        }
        __syncthreads();
    }
    if (cx < box.Bx && cy < box.By && cz < box.Bz) {
        const size_t c = ((size_t)cz * box.By + cy) * box.Bx + cx;
        ba.h[c] = ax;
        ba.h[box.nbox + c] = ay;
        ba.h[2 * box.nbox + c] = az;
    }
}

// ---------------------------------------------------------------------------
cudaError_t launch_particle(const Geom &g, const BodyConst &bc, DevState *st, cudaStream_t s) {
    k_particle<<<1, 32, 0, s>>>(g, bc, st);
    return cudaGetLastError();
}

cudaError_t launch_markers(const Geom &g, const BodyConst &bc, const BoxGeom &box, DevState *st, MarkerArrays m,
                           cudaStream_t s) {
    k_markers<<<(bc.nm + 127) / 128, 128, 0, s>>>(g, bc, box, st, m);
    return cudaGetLastError();
}

cudaError_t launch_bin(const BoxGeom &box, int nm, const int *bb, int *tile_list, int *tile_count, int cap,
                       cudaStream_t s) {
    k_bin<<<box.tx * box.ty * box.tz, 256, 0, s>>>(box, nm, bb, tile_list, tile_count, cap);
    return cudaGetLastError();
}

cudaError_t launch_interp(const BoxGeom &box, int nm, MarkerArrays m, BoxArrays ba, int mode, cudaStream_t s) {
    const long long threads = (long long)nm * 32;
    k_interp<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(box, nm, m, ba, mode);
    return cudaGetLastError();
}

cudaError_t launch_reduce_ft(int nm, MarkerArrays m, double *partials, DevState *st, cudaStream_t s) {
    k_reduce_ft<<<REDUCE_BLOCKS, 256, 0, s>>>(nm, m.ft, partials, st);
    return cudaGetLastError();
}

cudaError_t launch_spread(const BoxGeom &box, int nm, MarkerArrays m, BoxArrays ba, const int *tile_list,
                          const int *tile_count, int cap, cudaStream_t s) {
    k_spread<<<box.tx * box.ty * box.tz, 512, 0, s>>>(box, nm, m, ba, tile_list, tile_count, cap);
    return cudaGetLastError();
}

}  // namespace turret
