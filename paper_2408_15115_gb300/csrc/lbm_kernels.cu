// lbm_kernels.cu -- fused recursive-regularized D3Q27 collide+stream (pull)
// and the small passes that share its streaming and moment code.
//
// Method (Sec. 2.1 and Appendix A of arXiv 2408.15115): the post-collision
// populations are f* = f0(rho, u) + (1 - 1/tau) f1 (Eq. 7), with f0 the
// Hermite equilibrium carrying every D3Q27-supported term up to H6_xxyyzz and
// f1 the off-equilibrium part rebuilt from P1 = sum xi xi (f - f0) through the
// recursive coefficients a1^(n) (Eq. A.3).  Forcing follows the equilibrium
// velocity shift of Eq. 15 (reading: regularized BGK form, see turret.h).
//
// GB300 formulation (not the paper's): both f0 and f1 live in the 27-term
// tensor-product Hermite basis H_p(xi_x) H_q(xi_y) H_r(xi_z), p,q,r <= 2,
// which is orthogonal under the D3Q27 weights.  A collision is therefore
//   moments  : 3 separable passes of 3-point sums over x, y, z  (10 moments)
//   collision: C_pqr = rho u^p u^q u^r + (1 - 1/tau) a1_pqr, where
//              a1_pqr = 1/2 sum_ab P1_ab d^2(u^p u^q u^r)/du_a du_b
//              (the closed form of the recursion: a sum over index pairs)
//   rebuild  : 3 separable passes of 3x3 transforms with the weighted
//              basis g_p(xi) = w1(xi) H_p(xi)
// about 450 FP32 flops per cell.  Populations are stored as deviations
// q_i = f_i - w_i (FP32) or q_i / w_i scaled (FP16/BF16); the moments use
// drho = sum q, so no O(1) term cancels in single precision.
//
// Memory: SoA planes [27][z][y][x], one thread per cell, x fastest; each warp
// reads 27 coalesced 128-byte rows (the +-1 x-shifts hit the same sectors in
// L1/L2) and writes 27 aligned rows.  216 B/cell of HBM traffic in FP32.  The
// z index goes through the ring offset of the sliding window.
#include "turret_internal.cuh"

namespace turret {

__device__ __forceinline__ int zphys(int zl, int ring, int nz) {
    int z = zl + ring;
    return z >= nz ? z - nz : z;
}

__device__ __forceinline__ float tau_of(const Geom &g, int zl) {
    if (g.sponge > 0 && zl >= g.nz - g.sponge)
        return g.tau0 + (1.0f - g.tau0) * (float)(zl - (g.nz - g.sponge) + 1) / (float)g.sponge;
    return g.tau0;
}

// Source coordinate along one axis for velocity index e (= xi + 1): returns
// 0 (s valid, wrapped if periodic) or 1 (bounce-back through a no-slip face).
__device__ __forceinline__ int src_axis(int c, int e, int n, int bc, int &s) {
    s = c - (e - 1);
    if (s < 0) {
        if (bc == BC_PERIODIC) { s += n; return 0; }
        return 1;
    }
    if (s >= n) {
        if (bc == BC_PERIODIC) { s -= n; return 0; }
        return 1;
    }
    return 0;
}

// Deviation of the rest-density equilibrium f0_i(1, u) - w_i from the
// product form prod_a w1 [1 + 3 xi u + 9/2 (xi^2 - 1/3) u^2] (equal to the
// appendix equilibrium on D3Q27), expanded so the leading 1 cancels exactly.
__device__ __forceinline__ float eqfac_m1(int e, float u) {
    return e == 1 ? -1.5f * u * u : (e == 2 ? (3.0f * u + 3.0f * u * u) : (-3.0f * u + 3.0f * u * u));
}
__device__ __forceinline__ float ghost_dev(int i, float ux, float uy, float uz) {
    float a = eqfac_m1(i % 3, ux), b = eqfac_m1((i / 3) % 3, uy), c = eqfac_m1(i / 9, uz);
    return wq(i) * (a + b + c + a * b + a * c + b * c + a * b * c);
}

// Pull the 27 pre-collision deviations of cell (x, y, zl) from the
// post-collision buffer: f_i(x) = f*_i(x - xi_i); no-slip faces bounce back
// (halfway), the pressure top reads the ghost equilibrium, periodic faces wrap.
template <int ST>
__device__ __forceinline__ void pull27(const Geom &g, const typename Codec<ST>::T *__restrict__ f, int x, int y,
                                       int zl, int ring, const float *__restrict__ utop, float q[27]) {
    int sx[3], sy[3], szp[3], bxf[3], byf[3], bzf[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        bxf[e] = src_axis(x, e, g.nx, g.bc_x, sx[e]);
        byf[e] = src_axis(y, e, g.ny, g.bc_y, sy[e]);
        int zs = zl - (e - 1);
        bzf[e] = 0;
        if (zs < 0) {
            if (g.bc_bottom == BC_PERIODIC) zs += g.nz; else bzf[e] = 1;
        } else if (zs >= g.nz) {
            if (g.bc_top == BC_PERIODIC) zs -= g.nz;
            else bzf[e] = (g.bc_top == BC_PRESSURE) ? 2 : 1;
        }
        szp[e] = bzf[e] ? 0 : zphys(zs, ring, g.nz);
    }
    const size_t own = (size_t)zphys(zl, ring, g.nz) * g.plane + (size_t)y * g.nx + x;
#pragma unroll
    for (int ez = 0; ez < 3; ++ez)
#pragma unroll
        for (int ey = 0; ey < 3; ++ey)
#pragma unroll
            for (int ex = 0; ex < 3; ++ex) {
                const int i = ex + 3 * ey + 9 * ez;
                if (bxf[ex] == 1 || byf[ey] == 1 || bzf[ez] == 1) {
                    q[i] = Codec<ST>::load(f + (size_t)(26 - i) * g.ncell + own, 26 - i);
                } else if (bzf[ez] == 2) {
                    const size_t c = (size_t)sy[ey] * g.nx + sx[ex];
                    q[i] = ghost_dev(i, __ldg(utop + c), __ldg(utop + g.plane + c), __ldg(utop + 2 * g.plane + c));
                } else {
                    q[i] = Codec<ST>::load(
                        f + (size_t)i * g.ncell + (size_t)szp[ez] * g.plane + (size_t)sy[ey] * g.nx + sx[ex], i);
                }
            }
}

// Raw moments of the deviations up to second order: drho = sum q,
// j = sum xi q, Pi'_ab = sum xi_a xi_b q, by three separable 3-point passes.
struct Mom {
    float drho, jx, jy, jz, pxx, pyy, pzz, pxy, pxz, pyz;
};

__device__ __forceinline__ Mom moments27(const float q[27]) {
    float A0[9], A1[9], A2[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {  // k = ey + 3 ez; x pass
        const float a = q[3 * k], b = q[3 * k + 1], c = q[3 * k + 2];
        A0[k] = a + b + c;
        A1[k] = c - a;
        A2[k] = c + a;
    }
    float B00[3], B01[3], B02[3], B10[3], B11[3], B20[3];
#pragma unroll
    for (int ez = 0; ez < 3; ++ez) {  // y pass
        const int k = 3 * ez;
        B00[ez] = A0[k] + A0[k + 1] + A0[k + 2];
        B01[ez] = A0[k + 2] - A0[k];
        B02[ez] = A0[k + 2] + A0[k];
        B10[ez] = A1[k] + A1[k + 1] + A1[k + 2];
        B11[ez] = A1[k + 2] - A1[k];
        B20[ez] = A2[k] + A2[k + 1] + A2[k + 2];
    }
    Mom m;  // z pass
    m.drho = B00[0] + B00[1] + B00[2];
    m.jz = B00[2] - B00[0];
    m.pzz = B00[2] + B00[0];
    m.jy = B01[0] + B01[1] + B01[2];
    m.pyz = B01[2] - B01[0];
    m.pyy = B02[0] + B02[1] + B02[2];
    m.jx = B10[0] + B10[1] + B10[2];
    m.pxz = B10[2] - B10[0];
    m.pxy = B11[0] + B11[1] + B11[2];
    m.pxx = B20[0] + B20[1] + B20[2];
    return m;
}

// Macroscopic quantities from the deviation moments:
//   rho = 1 + drho, u = j / rho,
//   P1 = Pi - rho (I/3 + u u) = Pi' - drho I / 3 - j u^T.
struct Macro {
    float drho, rho, ux, uy, uz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz;
};

__device__ __forceinline__ Macro macro_of(const Mom &m) {
    Macro M;
    M.drho = m.drho;
    M.rho = 1.0f + m.drho;
    const float ir = 1.0f / M.rho;
    M.ux = m.jx * ir;
    M.uy = m.jy * ir;
    M.uz = m.jz * ir;
    const float d3 = m.drho * (1.0f / 3.0f);
    M.Pxx = m.pxx - d3 - m.jx * M.ux;
    M.Pyy = m.pyy - d3 - m.jy * M.uy;
    M.Pzz = m.pzz - d3 - m.jz * M.uz;
    M.Pxy = m.pxy - m.jx * M.uy;
    M.Pxz = m.pxz - m.jx * M.uz;
    M.Pyz = m.pyz - m.jy * M.uz;
    return M;
}

// Post-collision Hermite coefficients C[p + 3q + 9r] (deviation: C_000 - 1).
// forced: equilibrium part (1-w) rho m(u) + w rho m(u + tau h)  (scheme 0) or
// rho m(u + tau h) (scheme 1), m = monomial u_x^p u_y^q u_z^r.
__device__ __forceinline__ void collide_coeffs(const Macro &M, float omega, float tau, bool forced, float hx,
                                               float hy, float hz, int scheme, float C[27]) {
    const float px[3] = {1.0f, M.ux, M.ux * M.ux};
    const float py[3] = {1.0f, M.uy, M.uy * M.uy};
    const float pz[3] = {1.0f, M.uz, M.uz * M.uz};
    float ce[27];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int p = 0; p < 3; ++p) ce[p + 3 * q + 9 * r] = M.rho * px[p] * py[q] * pz[r];
    if (forced) {
        const float vx = M.ux + tau * hx, vy = M.uy + tau * hy, vz = M.uz + tau * hz;
        const float qx[3] = {1.0f, vx, vx * vx};
        const float qy[3] = {1.0f, vy, vy * vy};
        const float qz[3] = {1.0f, vz, vz * vz};
        const float a = (scheme == 1) ? 0.0f : (1.0f - omega);
        const float b = (scheme == 1) ? 1.0f : omega;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    const int k = p + 3 * q + 9 * r;
                    ce[k] = a * ce[k] + b * (M.rho * qx[p] * qy[q] * qz[r]);
                }
    }
    const float om1 = 1.0f - omega;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                // a1_pqr: half the P1-weighted Hessian of the monomial u^p u^q u^r
                float a1 = 0.0f;
                if (p == 2) a1 += M.Pxx * py[q] * pz[r];
                if (q == 2) a1 += M.Pyy * px[p] * pz[r];
                if (r == 2) a1 += M.Pzz * px[p] * py[q];
                if (p > 0 && q > 0) a1 += (float)(p * q) * M.Pxy * px[p - 1] * py[q - 1] * pz[r];
                if (p > 0 && r > 0) a1 += (float)(p * r) * M.Pxz * px[p - 1] * py[q] * pz[r - 1];
                if (q > 0 && r > 0) a1 += (float)(q * r) * M.Pyz * px[p] * py[q - 1] * pz[r - 1];
                const int k = p + 3 * q + 9 * r;
                C[k] = ce[k] + om1 * a1;
            }
    C[0] = M.drho;  // rho - 1: only deviations are stored
}

// Rebuild q_i = sum_pqr C_pqr g_p(xi_x) g_q(xi_y) g_r(xi_z) in place, with the
// weighted 1-D basis g(-1) = (1/6, -1/2, 1/2), g(0) = (2/3, 0, -1), g(+1) = (1/6, 1/2, 1/2).
__device__ __forceinline__ void tri(float &c0, float &c1, float &c2) {
    const float t = c0 * (1.0f / 6.0f) + 0.5f * c2;
    const float s = 0.5f * c1;
    const float mid = c0 * (2.0f / 3.0f) - c2;
    c0 = t - s;
    c1 = mid;
    c2 = t + s;
}
__device__ __forceinline__ void rebuild27(float C[27]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) tri(C[k], C[k + 9], C[k + 18]);  // z: stride 9
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int p = 0; p < 3; ++p) tri(C[p + 9 * r], C[p + 3 + 9 * r], C[p + 6 + 9 * r]);  // y: stride 3
#pragma unroll
    for (int k = 0; k < 9; ++k) tri(C[3 * k], C[3 * k + 1], C[3 * k + 2]);  // x: stride 1
}

// Wrapped offset of window coordinate c from box origin lo along one axis.
__device__ __forceinline__ int box_rel(int c, int lo, int n, bool periodic) {
    int r = c - lo;
    if (periodic) {
        r %= n;
        if (r < 0) r += n;
    }
    return r;
}

// ---------------------------------------------------------------------------
// K1: fused collide + stream over every cell of the window.
template <int ST, bool BOX>
__global__ void __launch_bounds__(128) k_collide_stream(Geom g, const typename Codec<ST>::T *__restrict__ src,
                                                        typename Codec<ST>::T *__restrict__ dst,
                                                        const float *__restrict__ utop_in,
                                                        float *__restrict__ utop_out,
                                                        const DevState *__restrict__ st,
                                                        const float *__restrict__ hbox, BoxGeom box) {
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 4 + threadIdx.y;
    const int zl = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int ring = st->ring;
    float q[27];
    pull27<ST>(g, src, x, y, zl, ring, utop_in, q);
    const float tau = tau_of(g, zl);
    const float omega = 1.0f / tau;
    bool forced = false;
    float hx = 0.0f, hy = 0.0f, hz = 0.0f;
    if (BOX) {
        const int rx = box_rel(x, st->box_lo[0], g.nx, g.bc_x == BC_PERIODIC);
        const int ry = box_rel(y, st->box_lo[1], g.ny, g.bc_y == BC_PERIODIC);
        const int rz = box_rel(zl, st->box_lo[2], g.nz, g.bc_bottom == BC_PERIODIC);
        if ((unsigned)rx < (unsigned)box.Bx && (unsigned)ry < (unsigned)box.By && (unsigned)rz < (unsigned)box.Bz) {
            const size_t b = ((size_t)rz * box.By + ry) * box.Bx + rx;
            hx = __ldg(hbox + b);
            hy = __ldg(hbox + box.nbox + b);
            hz = __ldg(hbox + 2 * box.nbox + b);
            forced = true;
        }
    }
    const Macro M = macro_of(moments27(q));
    if (zl == g.nz - 1) {
        const size_t c = (size_t)y * g.nx + x;
        utop_out[c] = M.ux;
        utop_out[g.plane + c] = M.uy;
        utop_out[2 * g.plane + c] = M.uz;
    }
    float C[27];
    collide_coeffs(M, omega, tau, forced, hx, hy, hz, g.force_scheme, C);
    rebuild27(C);
    const size_t own = (size_t)zphys(zl, ring, g.nz) * g.plane + (size_t)y * g.nx + x;
#pragma unroll
    for (int i = 0; i < 27; ++i) Codec<ST>::store(dst + (size_t)i * g.ncell + own, C[i], i);
}

// Equilibrium of given (rho - 1, u) fields (doubles, window order) as the
// post-collision state; u of the top plane goes to the pressure-ghost buffer.
template <int ST>
__global__ void k_init_equilibrium(Geom g, typename Codec<ST>::T *__restrict__ dst, const double *__restrict__ drho,
                                   const double *__restrict__ u, float *__restrict__ utop) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    const float dr = drho ? (float)drho[c] : 0.0f;
    Macro M;
    M.drho = dr;
    M.rho = (float)(1.0 + (drho ? drho[c] : 0.0));
    M.ux = u ? (float)u[3 * c] : 0.0f;
    M.uy = u ? (float)u[3 * c + 1] : 0.0f;
    M.uz = u ? (float)u[3 * c + 2] : 0.0f;
    M.Pxx = M.Pyy = M.Pzz = M.Pxy = M.Pxz = M.Pyz = 0.0f;
    float C[27];
    collide_coeffs(M, 1.0f, 1.0f, false, 0.0f, 0.0f, 0.0f, 0, C);
    rebuild27(C);
#pragma unroll
    for (int i = 0; i < 27; ++i) Codec<ST>::store(dst + (size_t)i * g.ncell + c, C[i], i);
    const long long z = c / g.plane;
    if (z == g.nz - 1) {
        const long long p = c - z * g.plane;
        utop[p] = M.ux;
        utop[g.plane + p] = M.uy;
        utop[2 * g.plane + p] = M.uz;
    }
}

// rho, u (or the 27 pre-collision deviations) of f(t) at every cell.
template <int ST>
__global__ void __launch_bounds__(128) k_macro(Geom g, const typename Codec<ST>::T *__restrict__ src,
                                               const float *__restrict__ utop_in, const DevState *__restrict__ st,
                                               float *__restrict__ out, int pops) {
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 4 + threadIdx.y;
    const int zl = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    float q[27];
    pull27<ST>(g, src, x, y, zl, st->ring, utop_in, q);
    const size_t c = ((size_t)zl * g.ny + y) * g.nx + x;
    if (pops) {
#pragma unroll
        for (int i = 0; i < 27; ++i) out[(size_t)i * g.ncell + c] = q[i];
        return;
    }
    const Macro M = macro_of(moments27(q));
    out[c] = M.rho;
    out[g.ncell + c] = M.ux;
    out[2 * g.ncell + c] = M.uy;
    out[3 * g.ncell + c] = M.uz;
}

// Window slide: the plane that enters the ring is reset to the rest state.
template <int ST>
__global__ void k_reseed(Geom g, typename Codec<ST>::T *__restrict__ dst, const DevState *__restrict__ st) {
    const int p = st->reseed_plane;
    if (p < 0) return;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.plane * 27) return;
    const long long i = c / g.plane, xy = c - i * g.plane;
    Codec<ST>::store(dst + (size_t)i * g.ncell + (size_t)p * g.plane + xy, 0.0f, (int)i);
}

// K2: u* and the stress of Eq. 10, sigma = -p I + (1/(2 tau) - 1) P1 with
// p = c_s^2 (rho - 1), at every support-box cell, from f(t+1) pulled from
// the post-collision buffer.  Box cells outside a closed face get zeros.
template <int ST>
__global__ void k_box_moments(Geom g, const typename Codec<ST>::T *__restrict__ src,
                              const float *__restrict__ utop_in, const DevState *__restrict__ st, BoxGeom box,
                              BoxArrays ba) {
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= box.nbox) return;
    const int bx = (int)(b % box.Bx);
    const int by = (int)((b / box.Bx) % box.By);
    const int bz = (int)(b / ((long long)box.Bx * box.By));
    int c[3] = {st->box_lo[0] + bx, st->box_lo[1] + by, st->box_lo[2] + bz};
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
        return;
    }
    float q[27];
    pull27<ST>(g, src, c[0], c[1], c[2], st->ring, utop_in, q);
    const Macro M = macro_of(moments27(q));
    const float tau = tau_of(g, c[2]);
    const float k2 = 0.5f / tau - 1.0f;
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
}

// ---------------------------------------------------------------------------
// Launchers.
static dim3 cell_grid(const Geom &g) { return dim3((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz); }

template <int ST>
static cudaError_t collide_t(const Geom &g, const void *src, void *dst, const float *utop_in, float *utop_out,
                             const DevState *st, const float *hbox, const BoxGeom &box, bool has_box,
                             cudaStream_t s) {
    using T = typename Codec<ST>::T;
    if (has_box)
        k_collide_stream<ST, true><<<cell_grid(g), dim3(32, 4), 0, s>>>(g, (const T *)src, (T *)dst, utop_in,
                                                                        utop_out, st, hbox, box);
    else
        k_collide_stream<ST, false><<<cell_grid(g), dim3(32, 4), 0, s>>>(g, (const T *)src, (T *)dst, utop_in,
                                                                         utop_out, st, hbox, box);
    return cudaGetLastError();
}

cudaError_t launch_collide_stream(const Geom &g, int storage, const void *src, void *dst, const float *utop_in,
                                  float *utop_out, const DevState *st, const float *hbox, const BoxGeom &box,
                                  bool has_box, cudaStream_t s) {
    switch (storage) {
        case ST_F32: return collide_t<ST_F32>(g, src, dst, utop_in, utop_out, st, hbox, box, has_box, s);
        case ST_F16: return collide_t<ST_F16>(g, src, dst, utop_in, utop_out, st, hbox, box, has_box, s);
        default: return collide_t<ST_BF16>(g, src, dst, utop_in, utop_out, st, hbox, box, has_box, s);
    }
}

cudaError_t launch_init_equilibrium(const Geom &g, int storage, void *dst, const double *drho, const double *u,
                                    float *utop, cudaStream_t s) {
    const unsigned nb = (unsigned)((g.ncell + 255) / 256);
    switch (storage) {
        case ST_F32: k_init_equilibrium<ST_F32><<<nb, 256, 0, s>>>(g, (float *)dst, drho, u, utop); break;
        case ST_F16: k_init_equilibrium<ST_F16><<<nb, 256, 0, s>>>(g, (__half *)dst, drho, u, utop); break;
        default: k_init_equilibrium<ST_BF16><<<nb, 256, 0, s>>>(g, (__nv_bfloat16 *)dst, drho, u, utop); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_macro(const Geom &g, int storage, const void *src, const float *utop_in, const DevState *st,
                         float *out, bool pops, cudaStream_t s) {
    switch (storage) {
        case ST_F32: k_macro<ST_F32><<<cell_grid(g), dim3(32, 4), 0, s>>>(g, (const float *)src, utop_in, st, out, pops); break;
        case ST_F16: k_macro<ST_F16><<<cell_grid(g), dim3(32, 4), 0, s>>>(g, (const __half *)src, utop_in, st, out, pops); break;
        default: k_macro<ST_BF16><<<cell_grid(g), dim3(32, 4), 0, s>>>(g, (const __nv_bfloat16 *)src, utop_in, st, out, pops); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_reseed(const Geom &g, int storage, void *dst, const DevState *st, cudaStream_t s) {
    const unsigned nb = (unsigned)((g.plane * 27 + 255) / 256);
    switch (storage) {
        case ST_F32: k_reseed<ST_F32><<<nb, 256, 0, s>>>(g, (float *)dst, st); break;
        case ST_F16: k_reseed<ST_F16><<<nb, 256, 0, s>>>(g, (__half *)dst, st); break;
        default: k_reseed<ST_BF16><<<nb, 256, 0, s>>>(g, (__nv_bfloat16 *)dst, st); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_box_moments(const Geom &g, int storage, const void *src, const float *utop_in,
                               const DevState *st, const BoxGeom &box, BoxArrays ba, cudaStream_t s) {
    const unsigned nb = (unsigned)((box.nbox + 127) / 128);
    switch (storage) {
        case ST_F32: k_box_moments<ST_F32><<<nb, 128, 0, s>>>(g, (const float *)src, utop_in, st, box, ba); break;
        case ST_F16: k_box_moments<ST_F16><<<nb, 128, 0, s>>>(g, (const __half *)src, utop_in, st, box, ba); break;
        default: k_box_moments<ST_BF16><<<nb, 128, 0, s>>>(g, (const __nv_bfloat16 *)src, utop_in, st, box, ba); break;
    }
    return cudaGetLastError();
}

}  // namespace turret
