// lbm_cell.cuh -- per-cell device code of the fused recursive-regularized
// D3Q27 collide+stream (pull) and of the passes that share its streaming and
// moment code; included by the single-run and the batched kernels, which thus
// run identical arithmetic.
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
// which is orthogonal under the D3Q27 weights.  The equilibrium coefficients
// are the monomials rho u_x^p u_y^q u_z^r and the recursive coefficients are
// a1_pqr = 1/2 sum_ab P1_ab d^2(u^p u^q u^r)/du_a du_b (the closed form of
// the recursion: a sum over index pairs), so every term is an outer product
// of one 3-vector per axis and a collision is
//   moments : 3 separable passes of 3-point sums over x, y, z (10 moments)
//   rebuild : per-axis factors X, X', X'' and 9 (y,z) pair terms, then
//             3 FMAs per population (collide_factored below)
// about 300 FP32 flops per cell.  Populations are stored as deviations
// s_i = 216 (f_i - w_i) (FP32) or s_i / W_i scaled (FP16/BF16) and every
// pass works in that storage domain (Codec); the moments use drho = sum s, so
// no O(1) term cancels in single precision.
//
// Memory: SoA planes [27][z][y][x], one thread per cell, x fastest; each warp
// reads 27 coalesced 128-byte rows (the +-1 x-shifts hit the same sectors in
// L1/L2) and writes 27 aligned rows.  216 B/cell of HBM traffic in FP32.  The
#pragma once
#include "turret_internal.cuh"

namespace turret {

// Stochastic rounding of BF16 stores (Geom::sround): the random bits come from
// the PCG hash of Jarzynski and Olano, "Hash Functions for GPU Rendering"
// (JCGT 9(3), 2020) -- a linear congruential step followed by O'Neill's PCG
// RXS-M-XS output permutation -- applied to a key made of the stored element's
// index and the time step, so a run is reproducible bit for bit.
__device__ __forceinline__ unsigned pcg_hash(unsigned v) {
    const unsigned state = v * 747796405u + 2891336453u;
    const unsigned word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}
__device__ __forceinline__ unsigned sr_key(int element, long long step) {
    return (unsigned)element + 0x9E3779B9u * (unsigned)step;
}
// bf16 bits of r with its magnitude rounded up with probability equal to the
// dropped fraction of the last kept bit (16 random bits added below the kept
// bits, then truncated): unbiased, E[stored] = r.
__device__ __forceinline__ void store_bf16_sr(__nv_bfloat16 *p, float r, unsigned rnd16) {
    *reinterpret_cast<unsigned short *>(p) = (unsigned short)((__float_as_uint(r) + rnd16) >> 16);
}

__device__ __forceinline__ int zphys(int zl, int ring, int nz) {
    int z = zl + ring;
    return z >= nz ? z - nz : z;
}

// Relaxation time of a logical plane (the sponge raises it linearly to 1 on
// the top plane); tabulated on the host in double precision.
__device__ __forceinline__ float tau_of(const Geom &g, int zl) { return __ldg(g.tau_z + zl); }
__device__ __forceinline__ float omega_of(const Geom &g, int zl) { return __ldg(g.omega_z + zl); }

// Source coordinate along one axis for velocity index e (= xi + 1) of a cell
// c in [0, n): returns 0 (s valid, wrapped if periodic) or 1 (bounce-back
// through a no-slip face).  Only xi = -1 can leave through the top face and
// only xi = +1 through the bottom one.
__device__ __forceinline__ int src_axis(int c, int e, int n, int bc, int &s) {
    if (e == 1) {
        s = c;
        return 0;
    }
    if (e == 0) {
        s = c + 1;
        if (s < n) return 0;
        s = 0;
        return bc == BC_PERIODIC ? 0 : 1;
    }
    s = c - 1;
    if (s >= 0) return 0;
    s = n - 1;
    return bc == BC_PERIODIC ? 0 : 1;
}

// Deviation of the rest-density equilibrium f0_i(1, u) - w_i from the
// product form prod_a w1 [1 + 3 xi u + 9/2 (xi^2 - 1/3) u^2] (equal to the
// appendix equilibrium on D3Q27), expanded so the leading 1 cancels exactly.
__device__ __forceinline__ float eqfac_m1(int e, float u) {
    return e == 1 ? -1.5f * u * u : (e == 2 ? (3.0f * u + 3.0f * u * u) : (-3.0f * u + 3.0f * u * u));
}
template <int ST>
__device__ __forceinline__ float ghost_dev(int i, float ux, float uy, float uz) {
    float a = eqfac_m1(i % 3, ux), b = eqfac_m1((i / 3) % 3, uy), c = eqfac_m1(i / 9, uz);
    const float w = Codec<ST>::scaled ? Codec<ST>::K : Wq(i);  // storage domain
    return w * (a + b + c + a * b + a * c + b * c + a * b * c);
}

// Pull the 27 pre-collision scaled deviations of cell (x, y, zl) from the
// post-collision buffer: f_i(x) = f*_i(x - xi_i); no-slip faces bounce back
// (halfway), the pressure top reads the ghost equilibrium, periodic faces wrap.
// A source on the plane that just entered the sliding window (reseed >= 0)
// holds stale data and reads as the rest equilibrium (deviation 0).
// The momentum a moving wall imparts to a population it bounces back,
// 2 w_i (xi_i . u_w) / c_s^2, in the storage domain: 6 W_i (xi . u_w) for the
// scaled deviations, 6 K (xi . u_w) for the scaled-by-weight forms.
template <int ST>
__device__ __forceinline__ float wall_term(int i, const float uw[3]) {
    const float xu = (float)(i % 3 - 1) * uw[0] + (float)((i / 3) % 3 - 1) * uw[1] + (float)(i / 9 - 1) * uw[2];
    return 6.0f * (Codec<ST>::scaled ? Codec<ST>::K : Wq(i)) * xu;
}

template <int ST>
__device__ __forceinline__ void pull27(const Geom &g, const typename Codec<ST>::T *__restrict__ f, int x, int y,
                                       int zl, int ring, int reseed, const float *__restrict__ utop, float q[27]) {
    int sx[3], sy[3], szp[3], bxf[3], byf[3], bzf[3], mvf[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        bxf[e] = src_axis(x, e, g.nx, g.bc_x, sx[e]);
        byf[e] = src_axis(y, e, g.ny, g.bc_y, sy[e]);
        int zs = zl - (e - 1);
        bzf[e] = 0;
        mvf[e] = 0;  // 1: the source lies beyond the moving bottom wall, 2: the moving top wall
        if (zs < 0) {
            if (g.bc_bottom == BC_PERIODIC) zs += g.nz; else bzf[e] = 1;
            if (g.bc_bottom == BC_MOVING) mvf[e] = 1;
        } else if (zs >= g.nz) {
            if (g.bc_top == BC_PERIODIC) zs -= g.nz;
            else bzf[e] = (g.bc_top == BC_PRESSURE) ? 2 : 1;
            if (g.bc_top == BC_MOVING) mvf[e] = 2;
        }
        szp[e] = bzf[e] ? 0 : zphys(zs, ring, g.nz);
        if (bzf[e] == 0 && szp[e] == reseed) bzf[e] = 3;
    }
    const int nx = g.nx, plane = (int)g.plane, ncell = (int)g.ncell;
    if ((bxf[0] | bxf[2] | byf[0] | byf[2] | bzf[0] | bzf[1] | bzf[2]) == 0) {
        // interior (or periodic) cell: 27 plain loads, each from one of nine
        // per-thread (x, y) column pointers plus a 32-bit offset (population,
        // plane) that is uniform over a block whose cells share z
        const typename Codec<ST>::T *P[3][3];
#pragma unroll
        for (int ey = 0; ey < 3; ++ey)
#pragma unroll
            for (int ex = 0; ex < 3; ++ex) P[ey][ex] = f + (sy[ey] * nx + sx[ex]);
#pragma unroll
        for (int ez = 0; ez < 3; ++ez)
#pragma unroll
            for (int ey = 0; ey < 3; ++ey)
#pragma unroll
                for (int ex = 0; ex < 3; ++ex) {
                    const int i = ex + 3 * ey + 9 * ez;
                    q[i] = Codec<ST>::load(P[ey][ex] + (i * ncell + szp[ez] * plane));
                }
        return;
    }
    const int zo = zphys(zl, ring, g.nz);
    const int own = zo * plane + y * nx + x;
    const bool own_rest = (zo == reseed);
#pragma unroll
    for (int ez = 0; ez < 3; ++ez)
#pragma unroll
        for (int ey = 0; ey < 3; ++ey)
#pragma unroll
            for (int ex = 0; ex < 3; ++ex) {
                const int i = ex + 3 * ey + 9 * ez;
                // (bounce-back: W_{26-i} = W_i, so the opposite population's stored
                // value is this one's in every storage domain)
                if (bxf[ex] == 1 || byf[ey] == 1 || bzf[ez] == 1) {
                    q[i] = own_rest ? 0.0f : Codec<ST>::load(f + (26 - i) * ncell + own);
                    if (mvf[ez]) q[i] += wall_term<ST>(i, mvf[ez] == 1 ? g.uw_bottom : g.uw_top);
                } else if (bzf[ez] == 3) {
                    q[i] = 0.0f;
                } else if (bzf[ez] == 2) {
                    const int c = sy[ey] * nx + sx[ex];
                    q[i] = ghost_dev<ST>(i, __ldg(utop + c), __ldg(utop + plane + c), __ldg(utop + 2 * plane + c));
                } else {
                    q[i] = Codec<ST>::load(f + i * ncell + szp[ez] * plane + sy[ey] * nx + sx[ex]);
                }
            }
}

// Raw moments of the scaled deviations up to second order (all times 216):
// drho = sum s, j = sum xi s, Pi'_ab = sum xi_a xi_b s, by three separable
// 3-point passes.  From a storage domain r_i = K s_i / W_i the passes carry
// the axis weights W1 = (1, 4, 1) of the sums that need them (the 4 sits on
// xi = 0, where the xi-weighted sums vanish anyway) and the result is
// divided by K (exact).
struct Mom {
    float drho, jx, jy, jz, pxx, pyy, pzz, pxy, pxz, pyz;
};

// a + W1(1) b + c: the centre weight applied in the storage domains
template <bool SC>
__device__ __forceinline__ float wsum3(float a, float b, float c) {
    return SC ? fmaf(4.0f, b, a + c) : a + b + c;
}

template <int ST>
__device__ __forceinline__ Mom moments27(const float q[27]) {
    constexpr bool SC = Codec<ST>::scaled;
    float A0[9], A1[9], A2[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {  // k = ey + 3 ez; x pass
        const float a = q[3 * k], b = q[3 * k + 1], c = q[3 * k + 2];
        A0[k] = wsum3<SC>(a, b, c);
        A1[k] = c - a;
        A2[k] = c + a;
    }
    float B00[3], B01[3], B02[3], B10[3], B11[3], B20[3];
#pragma unroll
    for (int ez = 0; ez < 3; ++ez) {  // y pass
        const int k = 3 * ez;
        B00[ez] = wsum3<SC>(A0[k], A0[k + 1], A0[k + 2]);
        B01[ez] = A0[k + 2] - A0[k];
        B02[ez] = A0[k + 2] + A0[k];
        B10[ez] = wsum3<SC>(A1[k], A1[k + 1], A1[k + 2]);
        B11[ez] = A1[k + 2] - A1[k];
        B20[ez] = wsum3<SC>(A2[k], A2[k + 1], A2[k + 2]);
    }
    Mom m;  // z pass
    m.drho = wsum3<SC>(B00[0], B00[1], B00[2]);
    m.jz = B00[2] - B00[0];
    m.pzz = B00[2] + B00[0];
    m.jy = wsum3<SC>(B01[0], B01[1], B01[2]);
    m.pyz = B01[2] - B01[0];
    m.pyy = wsum3<SC>(B02[0], B02[1], B02[2]);
    m.jx = wsum3<SC>(B10[0], B10[1], B10[2]);
    m.pxz = B10[2] - B10[0];
    m.pxy = wsum3<SC>(B11[0], B11[1], B11[2]);
    m.pxx = wsum3<SC>(B20[0], B20[1], B20[2]);
    if (SC && Codec<ST>::K != 1.0f) {
        constexpr float ik = 1.0f / Codec<ST>::K;
        m.drho *= ik; m.jx *= ik; m.jy *= ik; m.jz *= ik; m.pxx *= ik;
        m.pyy *= ik; m.pzz *= ik; m.pxy *= ik; m.pxz *= ik; m.pyz *= ik;
    }
    return m;
}

// Macroscopic quantities from the scaled moments (the tilde quantities are
// 216 times the physical ones):
//   drho = drho~ / 216, rho = 1 + drho, u = j~ / (216 + drho~),
//   P1~ = Pi'~ - drho~ I / 3 - j~ u^T   (= 216 [Pi - rho (I/3 + u u)]).
struct Macro {
    float drho, rho, ux, uy, uz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz;  // P: scaled by 216
};

__device__ __forceinline__ Macro macro_of(const Mom &m) {
    Macro M;
    M.drho = m.drho * INV_SCALE;
    M.rho = 1.0f + M.drho;
    const float ir = __frcp_rn(SCALE + m.drho);
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

// Per-axis factors of the collision.  With m(u) = prod_a u_a^{p_a} and the
// weighted basis g_p(xi) = w1(xi) H_p(xi), every term of the post-collision
// Hermite expansion is an outer product of one 3-vector per axis, so each
// population is rebuilt directly from per-axis vectors (here scaled by 6 so
// that the weights 6 w1 = (1, 4, 1) are exact):
//   X(e)   = 6 sum_p u^p g_p(e)      = W1(e) (1 + a(e)),  a = (-3u+3u^2, -3u^2/2, 3u+3u^2)
//   X'(e)  = 6 sum_p p u^(p-1) g_p(e) = (6u - 3, -12u, 6u + 3)
//   X''(e) = 6 sum_p p(p-1) u^(p-2) g_p(e) = (6, -12, 6)
// and, for P' = (1 - 1/tau) P1 (P1 the physical tensor),
//   s_i = 216 (f*_i - w_i) = [rho X Y Z - W_i] + X'' [P'xx/2 Y Z]
//         + X [P'yy/2 Y'' Z + P'zz/2 Y Z'' + P'yz Y' Z'] + X' [P'xy Y' Z + P'xz Y Z'],
// the bracketed equilibrium deviation evaluated as W_i (rho E + drho) with
// E = (1+a_x)(1+a_y)(1+a_z) - 1 expanded so no O(1) term cancels.  In the
// scaled storage domains every per-axis factor is divided by W1(e), which
// divides each product by W_i: X / W1 = 1 + a, X' / W1, X'' / W1 = (6, -3, 6).
struct AxisF {
    float a[3], X[3], Xp[3];
};

template <bool SC>
__device__ __forceinline__ AxisF axis_of(float u) {
    AxisF f;
    const float u2 = u * u;
    f.a[0] = 3.0f * (u2 - u);
    f.a[1] = -1.5f * u2;
    f.a[2] = 3.0f * (u2 + u);
    f.X[0] = 1.0f + f.a[0];
    f.X[1] = SC ? 1.0f + f.a[1] : 4.0f * (1.0f + f.a[1]);
    f.X[2] = 1.0f + f.a[2];
    f.Xp[0] = 6.0f * u - 3.0f;
    f.Xp[1] = SC ? -3.0f * u : -12.0f * u;
    f.Xp[2] = 6.0f * u + 3.0f;
    return f;
}

// Equilibrium deviation W_i (rho E + drho) (SC: rho E + drho), times c, into s.
template <bool SC>
__device__ __forceinline__ void add_eq_dev(const AxisF &fx, const AxisF &fy, const AxisF &fz, float rho,
                                           float drho, float c, float s[27], bool first) {
    float sxy[9];
#pragma unroll
    for (int ey = 0; ey < 3; ++ey)
#pragma unroll
        for (int ex = 0; ex < 3; ++ex) sxy[ex + 3 * ey] = fmaf(fx.a[ex], fy.a[ey], fx.a[ex] + fy.a[ey]);
#pragma unroll
    for (int ez = 0; ez < 3; ++ez)
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int i = k + 9 * ez;
            const float E = fmaf(sxy[k], fz.a[ez], sxy[k] + fz.a[ez]);
            const float v = (SC ? c : c * Wq(i)) * fmaf(E, rho, drho);
            s[i] = first ? v : s[i] + v;
        }
}

// The same for the unforced equilibrium, whose factor c = K is a power of two:
// K W_i (rho E + drho) = fma(E, K W_i rho, K W_i drho) bit for bit (scaling by
// a power of two is exact), one operation less per population.
template <bool SC>
__device__ __forceinline__ void set_eq_dev_pow2(const AxisF &fx, const AxisF &fy, const AxisF &fz, float rho,
                                                float drho, float K, float s[27]) {
    float r[4], d[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const float c = K * (float)(1 << (2 * w));  // K W for W = 1, 4, 16, 64
        r[w] = c * rho;
        d[w] = c * drho;
    }
    float sxy[9];
#pragma unroll
    for (int ey = 0; ey < 3; ++ey)
#pragma unroll
        for (int ex = 0; ex < 3; ++ex) sxy[ex + 3 * ey] = fmaf(fx.a[ex], fy.a[ey], fx.a[ex] + fy.a[ey]);
#pragma unroll
    for (int ez = 0; ez < 3; ++ez)
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int i = k + 9 * ez;
            const int lw = SC ? 0 : (i % 3 == 1) + ((i / 3) % 3 == 1) + (i / 9 == 1);  // log4 W_i
            const float E = fmaf(sxy[k], fz.a[ez], sxy[k] + fz.a[ez]);
            s[i] = fmaf(E, r[lw], d[lw]);
        }
}

// Post-collision populations of one cell in the storage domain of ST
// (FP32: s_i = 216 (f*_i - w_i)).  forced: equilibrium part
// (1-w) f0(u) + w f0(u + tau h) (scheme 0) or f0(u + tau h) (scheme 1), both
// reducing to f0(u) at h = 0.
template <int ST>
__device__ __forceinline__ void collide_factored(const Macro &M, float omega, float tau, bool forced, float hx,
                                                 float hy, float hz, int scheme, float s[27]) {
    constexpr bool SC = Codec<ST>::scaled;
    constexpr float K = Codec<ST>::K;
    const AxisF fx = axis_of<SC>(M.ux), fy = axis_of<SC>(M.uy), fz = axis_of<SC>(M.uz);
    if (!forced) {
        set_eq_dev_pow2<SC>(fx, fy, fz, M.rho, M.drho, K, s);
    } else {
        const AxisF vx = axis_of<SC>(M.ux + tau * hx), vy = axis_of<SC>(M.uy + tau * hy),
                    vz = axis_of<SC>(M.uz + tau * hz);
        if (scheme == 1) {
            add_eq_dev<SC>(vx, vy, vz, M.rho, M.drho, K, s, true);
        } else {
            add_eq_dev<SC>(fx, fy, fz, M.rho, M.drho, K * (1.0f - omega), s, true);
            add_eq_dev<SC>(vx, vy, vz, M.rho, M.drho, K * omega, s, false);
        }
    }
    // P' = (1 - 1/tau) P1 with P1 = P1~ / 216 (times K in the storage domain)
    const float om1 = (1.0f - omega) * (INV_SCALE * K);
    const float hxx = 0.5f * om1 * M.Pxx, hyy = 0.5f * om1 * M.Pyy, hzz = 0.5f * om1 * M.Pzz;
    const float pxy = om1 * M.Pxy, pxz = om1 * M.Pxz, pyz = om1 * M.Pyz;
    const float Xpp[3] = {6.0f, SC ? -3.0f : -12.0f, 6.0f};
    float cY[3], cZ[3], bY[3], aY[3], bZ[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        cY[e] = hyy * Xpp[e];     // P'yy/2 Y''
        cZ[e] = hzz * Xpp[e];     // P'zz/2 Z''
        bY[e] = pyz * fy.Xp[e];   // P'yz Y'
        aY[e] = pxy * fy.Xp[e];   // P'xy Y'
        bZ[e] = pxz * fz.Xp[e];   // P'xz Z'
    }
#pragma unroll
    for (int ez = 0; ez < 3; ++ez)
#pragma unroll
        for (int ey = 0; ey < 3; ++ey) {
            const float G0 = hxx * (fy.X[ey] * fz.X[ez]);
            const float G1 = fmaf(cY[ey], fz.X[ez], fmaf(fy.X[ey], cZ[ez], bY[ey] * fz.Xp[ez]));
            const float G2 = fmaf(aY[ey], fz.X[ez], fy.X[ey] * bZ[ez]);
#pragma unroll
            for (int ex = 0; ex < 3; ++ex) {
                const int i = ex + 3 * ey + 9 * ez;
                s[i] = fmaf(Xpp[ex], G0, fmaf(fx.X[ex], G1, fmaf(fx.Xp[ex], G2, s[i])));
            }
        }
}

// Offset of window coordinate c from (box origin - margin) along one axis,
// wrapped into [0, n) along periodic axes (lo_w: the origin already wrapped).
__device__ __forceinline__ int rel_axis(int c, int lo, int lo_w, int margin, int n, bool periodic) {
    if (!periodic) return c - lo + margin;
    int r = c - lo_w + margin;
    r += (r < 0) ? n : 0;
    r -= (r >= n) ? n : 0;
    return r;
}

// ---------------------------------------------------------------------------
// K1: fused collide + stream.  MODE selects the cells and the forcing:
//   K1_ALL    every cell, no support box (fluid without particle);
//   K1_ALLF   every cell, h_imm read on the support box;
//   K1_FAR    every cell outside the near region (support box grown by
//             NEAR_GROW cells) -- no forcing there;
//   K1_NEAR   the near region only (grid over its extent), with forcing.
// FAR and NEAR together cover the window once.
enum { K1_ALL = 0, K1_ALLF = 1, K1_FAR = 2, K1_NEAR = 3 };

// One cell of K1 (scalar arithmetic; the near-region launch, which is small
// and on the critical path, runs one cell per thread).  (cx, cy, cz): window
// coordinates (x, y, logical z) for ALL / ALLF / FAR, coordinates within the
// near region for NEAR; out-of-range coordinates return.  S is the window
// slot of the pulled time level.
template <int ST, int MODE>
__device__ __forceinline__ void k1_cell(const Geom &g, const typename Codec<ST>::T *__restrict__ src,
                                        typename Codec<ST>::T *__restrict__ dst, const float *__restrict__ utop_in,
                                        float *__restrict__ utop_out, const BodySlot &S,
                                        const float *__restrict__ hbox, const BoxGeom &box, int cx, int cy, int cz) {
    int x, y, zl;
    const bool perx = g.bc_x == BC_PERIODIC, pery = g.bc_y == BC_PERIODIC, perz = g.bc_bottom == BC_PERIODIC;
    if (MODE == K1_NEAR) {
        // grid over the near region; map to window cells, skip cells outside closed faces
        if (cx >= box.Bx + 2 * NEAR_GROW || cy >= box.By + 2 * NEAR_GROW) return;
        x = (perx ? S.box_lo_w[0] : S.box_lo[0]) - NEAR_GROW + cx;
        y = (pery ? S.box_lo_w[1] : S.box_lo[1]) - NEAR_GROW + cy;
        zl = (perz ? S.box_lo_w[2] : S.box_lo[2]) - NEAR_GROW + cz;
        if (perx) { x += (x < 0) ? g.nx : 0; x -= (x >= g.nx) ? g.nx : 0; } else if (x < 0 || x >= g.nx) return;
        if (pery) { y += (y < 0) ? g.ny : 0; y -= (y >= g.ny) ? g.ny : 0; } else if (y < 0 || y >= g.ny) return;
        if (perz) { zl += (zl < 0) ? g.nz : 0; zl -= (zl >= g.nz) ? g.nz : 0; } else if (zl < 0 || zl >= g.nz) return;
    } else {
        x = cx;
        y = cy;
        zl = cz;
        if (x >= g.nx || y >= g.ny) return;
        if (MODE == K1_FAR) {
            // the z test first: zl is the same for a whole block (plane)
            const int rz = rel_axis(zl, S.box_lo[2], S.box_lo_w[2], NEAR_GROW, g.nz, perz);
            if ((unsigned)rz < (unsigned)(box.Bz + 2 * NEAR_GROW)) {
                const int rx = rel_axis(x, S.box_lo[0], S.box_lo_w[0], NEAR_GROW, g.nx, perx);
                const int ry = rel_axis(y, S.box_lo[1], S.box_lo_w[1], NEAR_GROW, g.ny, pery);
                if ((unsigned)rx < (unsigned)(box.Bx + 2 * NEAR_GROW) &&
                    (unsigned)ry < (unsigned)(box.By + 2 * NEAR_GROW))
                    return;
            }
        }
    }
    const int ring = S.ring;
    float q[27];
    pull27<ST>(g, src, x, y, zl, ring, S.reseed, utop_in, q);
    const float omega = omega_of(g, zl);
    bool forced = false;
    float hx = 0.0f, hy = 0.0f, hz = 0.0f;
    if (MODE == K1_ALLF || MODE == K1_NEAR) {
        const int rx = rel_axis(x, S.box_lo[0], S.box_lo_w[0], 0, g.nx, perx);
        const int ry = rel_axis(y, S.box_lo[1], S.box_lo_w[1], 0, g.ny, pery);
        const int rz = rel_axis(zl, S.box_lo[2], S.box_lo_w[2], 0, g.nz, perz);
        if ((unsigned)rx < (unsigned)box.Bx && (unsigned)ry < (unsigned)box.By && (unsigned)rz < (unsigned)box.Bz) {
            const size_t b = ((size_t)rz * box.By + ry) * box.Bx + rx;
            hx = __ldg(hbox + b);
            hy = __ldg(hbox + box.nbox + b);
            hz = __ldg(hbox + 2 * box.nbox + b);
            forced = true;
        }
    }
    const Macro M = macro_of(moments27<ST>(q));
    if (zl == g.nz - 1) {
        const size_t c = (size_t)y * g.nx + x;
        utop_out[c] = M.ux;
        utop_out[g.plane + c] = M.uy;
        utop_out[2 * g.plane + c] = M.uz;
    }
    if (MODE == K1_ALLF || MODE == K1_NEAR)
        collide_factored<ST>(M, omega, tau_of(g, zl), forced, hx, hy, hz, g.force_scheme, q);
    else
        collide_factored<ST>(M, omega, 1.0f, false, 0.0f, 0.0f, 0.0f, 0, q);
    const int oz = zphys(zl, ring, g.nz) * (int)g.plane;
    const int ncell = (int)g.ncell;
    typename Codec<ST>::T *d = dst + (y * g.nx + x);
    if (ST == ST_BF16 && g.sround) {
        const int own = oz + y * g.nx + x;
#pragma unroll
        for (int i = 0; i < 27; ++i)
            store_bf16_sr(reinterpret_cast<__nv_bfloat16 *>(d + (i * ncell + oz)), q[i],
                          pcg_hash(sr_key(i * ncell + own, S.step)) & 0xffffu);
        return;
    }
#pragma unroll
    for (int i = 0; i < 27; ++i) Codec<ST>::store(d + (i * ncell + oz), q[i]);
}

// ---------------------------------------------------------------------------
// K1 on a pair of cells (x, y, z) and (x, y, z + 1) per thread.  Every FP32
// operation of the moments and the collision is issued once for both cells
// as a packed f32x2 instruction (per lane the same correctly rounded
// operation); the x/y source indices, boundary flags and region tests are
// shared.  A cell's result never depends on the other cell of its pair.
typedef float2 f2;
__device__ __forceinline__ f2 F2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 padd(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 psub(f2 a, f2 b) { return __ffma2_rn(b, F2(-1.0f), a); }  // exact product
__device__ __forceinline__ f2 pmul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 pfma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

template <bool SC>
__device__ __forceinline__ f2 pwsum3(f2 a, f2 b, f2 c) {
    return SC ? pfma(F2(4.0f), b, padd(a, c)) : padd(padd(a, b), c);
}

struct Mom2 {
    f2 drho, jx, jy, jz, pxx, pyy, pzz, pxy, pxz, pyz;
};

template <int ST>
__device__ __forceinline__ Mom2 moments27x2(const f2 q[27]) {
    constexpr bool SC = Codec<ST>::scaled;
    f2 A0[9], A1[9], A2[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const f2 a = q[3 * k], b = q[3 * k + 1], c = q[3 * k + 2];
        A0[k] = pwsum3<SC>(a, b, c);
        A1[k] = psub(c, a);
        A2[k] = padd(c, a);
    }
    f2 B00[3], B01[3], B02[3], B10[3], B11[3], B20[3];
#pragma unroll
    for (int ez = 0; ez < 3; ++ez) {
        const int k = 3 * ez;
        B00[ez] = pwsum3<SC>(A0[k], A0[k + 1], A0[k + 2]);
        B01[ez] = psub(A0[k + 2], A0[k]);
        B02[ez] = padd(A0[k + 2], A0[k]);
        B10[ez] = pwsum3<SC>(A1[k], A1[k + 1], A1[k + 2]);
        B11[ez] = psub(A1[k + 2], A1[k]);
        B20[ez] = pwsum3<SC>(A2[k], A2[k + 1], A2[k + 2]);
    }
    Mom2 m;
    m.drho = pwsum3<SC>(B00[0], B00[1], B00[2]);
    m.jz = psub(B00[2], B00[0]);
    m.pzz = padd(B00[2], B00[0]);
    m.jy = pwsum3<SC>(B01[0], B01[1], B01[2]);
    m.pyz = psub(B01[2], B01[0]);
    m.pyy = pwsum3<SC>(B02[0], B02[1], B02[2]);
    m.jx = pwsum3<SC>(B10[0], B10[1], B10[2]);
    m.pxz = psub(B10[2], B10[0]);
    m.pxy = pwsum3<SC>(B11[0], B11[1], B11[2]);
    m.pxx = pwsum3<SC>(B20[0], B20[1], B20[2]);
    if (SC && Codec<ST>::K != 1.0f) {
        const f2 ik = F2(1.0f / Codec<ST>::K);
        m.drho = pmul(m.drho, ik); m.jx = pmul(m.jx, ik); m.jy = pmul(m.jy, ik); m.jz = pmul(m.jz, ik);
        m.pxx = pmul(m.pxx, ik); m.pyy = pmul(m.pyy, ik); m.pzz = pmul(m.pzz, ik);
        m.pxy = pmul(m.pxy, ik); m.pxz = pmul(m.pxz, ik); m.pyz = pmul(m.pyz, ik);
    }
    return m;
}

struct Macro2 {
    f2 drho, rho, ux, uy, uz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz;  // P: scaled by 216
};

__device__ __forceinline__ Macro2 macro_of2(const Mom2 &m) {
    Macro2 M;
    M.drho = pmul(m.drho, F2(INV_SCALE));
    M.rho = padd(F2(1.0f), M.drho);
    const f2 den = padd(F2(SCALE), m.drho);
    const f2 ir = make_float2(__frcp_rn(den.x), __frcp_rn(den.y));
    M.ux = pmul(m.jx, ir);
    M.uy = pmul(m.jy, ir);
    M.uz = pmul(m.jz, ir);
    const f2 d3 = pmul(m.drho, F2(1.0f / 3.0f));
    M.Pxx = psub(psub(m.pxx, d3), pmul(m.jx, M.ux));
    M.Pyy = psub(psub(m.pyy, d3), pmul(m.jy, M.uy));
    M.Pzz = psub(psub(m.pzz, d3), pmul(m.jz, M.uz));
    M.Pxy = psub(m.pxy, pmul(m.jx, M.uy));
    M.Pxz = psub(m.pxz, pmul(m.jx, M.uz));
    M.Pyz = psub(m.pyz, pmul(m.jy, M.uz));
    return M;
}

struct AxisF2 {
    f2 a[3], X[3], Xp[3];
};

template <bool SC>
__device__ __forceinline__ AxisF2 axis_of2(f2 u) {
    AxisF2 f;
    const f2 u2 = pmul(u, u);
    f.a[0] = pmul(F2(3.0f), psub(u2, u));
    f.a[1] = pmul(F2(-1.5f), u2);
    f.a[2] = pmul(F2(3.0f), padd(u2, u));
    f.X[0] = padd(F2(1.0f), f.a[0]);
    f.X[1] = SC ? padd(F2(1.0f), f.a[1]) : pmul(F2(4.0f), padd(F2(1.0f), f.a[1]));
    f.X[2] = padd(F2(1.0f), f.a[2]);
    f.Xp[0] = pfma(F2(6.0f), u, F2(-3.0f));
    f.Xp[1] = pmul(F2(SC ? -3.0f : -12.0f), u);
    f.Xp[2] = pfma(F2(6.0f), u, F2(3.0f));
    return f;
}

// c * W_i (rho E + drho) (SC: c (rho E + drho)) into s, or added to s; c per lane.
template <bool SC>
__device__ __forceinline__ void add_eq_dev2(const AxisF2 &fx, const AxisF2 &fy, const AxisF2 &fz, f2 rho, f2 drho,
                                            f2 c, f2 s[27], bool first) {
    f2 cw[4];  // c W for W = 1, 4, 16, 64
    cw[0] = c;
    if (!SC) {
        cw[1] = pmul(c, F2(4.0f));
        cw[2] = pmul(c, F2(16.0f));
        cw[3] = pmul(c, F2(64.0f));
    }
    f2 sxy[9];
#pragma unroll
    for (int ey = 0; ey < 3; ++ey)
#pragma unroll
        for (int ex = 0; ex < 3; ++ex) sxy[ex + 3 * ey] = pfma(fx.a[ex], fy.a[ey], padd(fx.a[ex], fy.a[ey]));
#pragma unroll
    for (int ez = 0; ez < 3; ++ez)
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int i = k + 9 * ez;
            const int lw = (i % 3 == 1) + ((i / 3) % 3 == 1) + (i / 9 == 1);  // log4 W_i
            const f2 E = pfma(sxy[k], fz.a[ez], padd(sxy[k], fz.a[ez]));
            const f2 v = pmul(SC ? c : cw[lw], pfma(E, rho, drho));
            s[i] = first ? v : padd(s[i], v);
        }
}

// set_eq_dev_pow2 for a cell pair: the unforced equilibrium deviation
// K W_i (rho E + drho) as fma(E, K W_i rho, K W_i drho), bit for bit equal.
template <bool SC>
__device__ __forceinline__ void set_eq_dev2_pow2(const AxisF2 &fx, const AxisF2 &fy, const AxisF2 &fz, f2 rho,
                                                 f2 drho, float K, f2 s[27]) {
    f2 r[4], d[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        if (SC && w > 0) continue;
        const f2 c = F2(K * (float)(1 << (2 * w)));  // K W for W = 1, 4, 16, 64
        r[w] = pmul(c, rho);
        d[w] = pmul(c, drho);
    }
    f2 sxy[9];
#pragma unroll
    for (int ey = 0; ey < 3; ++ey)
#pragma unroll
        for (int ex = 0; ex < 3; ++ex) sxy[ex + 3 * ey] = pfma(fx.a[ex], fy.a[ey], padd(fx.a[ex], fy.a[ey]));
#pragma unroll
    for (int ez = 0; ez < 3; ++ez)
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int i = k + 9 * ez;
            const int lw = SC ? 0 : (i % 3 == 1) + ((i / 3) % 3 == 1) + (i / 9 == 1);  // log4 W_i
            const f2 E = pfma(sxy[k], fz.a[ez], padd(sxy[k], fz.a[ez]));
            s[i] = pfma(E, r[lw], d[lw]);
        }
}

// Post-collision populations of two cells in the storage domain of ST.
// forced lanes take (1-w) f0(u) + w f0(u + tau h) (scheme 0) or
// f0(u + tau h) (scheme 1); other lanes f0(u) (their h is zero, and their
// scheme-0 weights are 1 and 0, so the shifted term adds an exact zero).
template <int ST>
__device__ __forceinline__ void collide_pair(const Macro2 &M, f2 omega, f2 tau, bool anyforced, bool fa, bool fb,
                                             f2 h[3], int scheme, f2 s[27]) {
    constexpr bool SC = Codec<ST>::scaled;
    constexpr float K = Codec<ST>::K;
    const AxisF2 fx = axis_of2<SC>(M.ux), fy = axis_of2<SC>(M.uy), fz = axis_of2<SC>(M.uz);
    if (!anyforced) {
        set_eq_dev2_pow2<SC>(fx, fy, fz, M.rho, M.drho, K, s);
    } else {
        const AxisF2 vx = axis_of2<SC>(pfma(tau, h[0], M.ux)), vy = axis_of2<SC>(pfma(tau, h[1], M.uy)),
                     vz = axis_of2<SC>(pfma(tau, h[2], M.uz));
        if (scheme == 1) {
            add_eq_dev2<SC>(vx, vy, vz, M.rho, M.drho, F2(K), s, true);
        } else {
            const f2 w1 = pmul(F2(K), psub(F2(1.0f), omega)), w2 = pmul(F2(K), omega);
            const f2 c1 = make_float2(fa ? w1.x : K, fb ? w1.y : K);
            const f2 c2 = make_float2(fa ? w2.x : 0.0f, fb ? w2.y : 0.0f);
            add_eq_dev2<SC>(fx, fy, fz, M.rho, M.drho, c1, s, true);
            add_eq_dev2<SC>(vx, vy, vz, M.rho, M.drho, c2, s, false);
        }
    }
    const f2 om1 = pmul(psub(F2(1.0f), omega), F2(INV_SCALE * K));
    const f2 hom = pmul(F2(0.5f), om1);
    const f2 hxx = pmul(hom, M.Pxx), hyy = pmul(hom, M.Pyy), hzz = pmul(hom, M.Pzz);
    const f2 pxy = pmul(om1, M.Pxy), pxz = pmul(om1, M.Pxz), pyz = pmul(om1, M.Pyz);
    const float xpp[3] = {6.0f, SC ? -3.0f : -12.0f, 6.0f};
    f2 cY[3], cZ[3], bY[3], aY[3], bZ[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        cY[e] = pmul(hyy, F2(xpp[e]));
        cZ[e] = pmul(hzz, F2(xpp[e]));
        bY[e] = pmul(pyz, fy.Xp[e]);
        aY[e] = pmul(pxy, fy.Xp[e]);
        bZ[e] = pmul(pxz, fz.Xp[e]);
    }
#pragma unroll
    for (int ez = 0; ez < 3; ++ez)
#pragma unroll
        for (int ey = 0; ey < 3; ++ey) {
            const f2 G0 = pmul(hxx, pmul(fy.X[ey], fz.X[ez]));
            const f2 G1 = pfma(cY[ey], fz.X[ez], pfma(fy.X[ey], cZ[ez], pmul(bY[ey], fz.Xp[ez])));
            const f2 G2 = pfma(aY[ey], fz.X[ez], pmul(fy.X[ey], bZ[ez]));
#pragma unroll
            for (int ex = 0; ex < 3; ++ex) {
                const int i = ex + 3 * ey + 9 * ez;
                s[i] = pfma(F2(xpp[ex]), G0, pfma(fx.X[ex], G1, pfma(fx.Xp[ex], G2, s[i])));
            }
        }
}

// Source plane of logical plane zl for velocity index ez (= xi_z + 1): 0 and
// the physical plane, 1 bounce-back, 2 pressure ghost, 3 the entering plane.
__device__ __forceinline__ int src_z(const Geom &g, int zl, int ez, int ring, int reseed, int &sz) {
    int zs = zl - (ez - 1), flag = 0;
    if (zs < 0) {
        if (g.bc_bottom == BC_PERIODIC) zs += g.nz; else flag = 1;
    } else if (zs >= g.nz) {
        if (g.bc_top == BC_PERIODIC) zs -= g.nz;
        else flag = (g.bc_top == BC_PRESSURE) ? 2 : 1;
    }
    sz = flag ? 0 : zphys(zs, ring, g.nz);
    if (flag == 0 && sz == reseed) flag = 3;
    return flag;
}

// Pull the 27 populations of two cells (x, y, za) and (x, y, zb) (window
// coordinates, both inside the window); interior and periodic pairs take 54
// plain loads, any other pair the per-cell rule of pull27.
template <int ST>
__device__ __forceinline__ void pull27x2(const Geom &g, const typename Codec<ST>::T *__restrict__ f, int x, int y,
                                         int za, int zb, int ring, int reseed, const float *__restrict__ utop,
                                         f2 q[27]) {
    int sx[3], sy[3], bxf[3], byf[3], sa[3], sb[3], ba[3], bb[3];
    int flags = 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        bxf[e] = src_axis(x, e, g.nx, g.bc_x, sx[e]);
        byf[e] = src_axis(y, e, g.ny, g.bc_y, sy[e]);
        ba[e] = src_z(g, za, e, ring, reseed, sa[e]);
        bb[e] = src_z(g, zb, e, ring, reseed, sb[e]);
        flags |= bxf[e] | byf[e] | ba[e] | bb[e];
    }
    const int nx = g.nx, plane = (int)g.plane, ncell = (int)g.ncell;  // 27 ncell < 2^31
    if (flags == 0) {
        // nine per-thread (x, y) column pointers; the (population, plane)
        // offsets are uniform over a block whose pairs share z
        const typename Codec<ST>::T *P[3][3];
#pragma unroll
        for (int ey = 0; ey < 3; ++ey)
#pragma unroll
            for (int ex = 0; ex < 3; ++ex) P[ey][ex] = f + (sy[ey] * nx + sx[ex]);
#pragma unroll
        for (int ez = 0; ez < 3; ++ez) {
            const int oa = sa[ez] * plane, ob = sb[ez] * plane;
#pragma unroll
            for (int ey = 0; ey < 3; ++ey)
#pragma unroll
                for (int ex = 0; ex < 3; ++ex) {
                    const int i = ex + 3 * ey + 9 * ez;
                    q[i].x = Codec<ST>::load(P[ey][ex] + (i * ncell + oa));
                    q[i].y = Codec<ST>::load(P[ey][ex] + (i * ncell + ob));
                }
        }
        return;
    }
    float qa[27];
    pull27<ST>(g, f, x, y, za, ring, reseed, utop, qa);
#pragma unroll
    for (int i = 0; i < 27; ++i) q[i].x = qa[i];
    pull27<ST>(g, f, x, y, zb, ring, reseed, utop, qa);
#pragma unroll
    for (int i = 0; i < 27; ++i) q[i].y = qa[i];
}

template <int ST, int MODE, bool STORE = true>
__device__ __forceinline__ void k1_pair_collide_store(const Geom &g, typename Codec<ST>::T *__restrict__ dst,
                                                      float *__restrict__ utop_out, const BodySlot &S,
                                                      const float *__restrict__ hbox, const BoxGeom &box, int x,
                                                      int y, const int z[2], const bool on[2], f2 q[27]);

// K1 for the cell pair (cx, cy, cz), (cx, cy, cz + 1): window coordinates for
// ALL / ALLF / FAR, near-region coordinates for NEAR; cells outside the
// window (or the mode's region) are not written, and a pair with none
// inside returns.
template <int ST, int MODE>
__device__ __forceinline__ void k1_pair(const Geom &g, const typename Codec<ST>::T *__restrict__ src,
                                        typename Codec<ST>::T *__restrict__ dst, const float *__restrict__ utop_in,
                                        float *__restrict__ utop_out, const BodySlot &S,
                                        const float *__restrict__ hbox, const BoxGeom &box, int cx, int cy, int cz) {
    const bool perx = g.bc_x == BC_PERIODIC, pery = g.bc_y == BC_PERIODIC, perz = g.bc_bottom == BC_PERIODIC;
    int x, y, z[2];
    bool on[2];
    if (MODE == K1_NEAR) {
        if (cx >= box.Bx + 2 * NEAR_GROW || cy >= box.By + 2 * NEAR_GROW) return;
        x = (perx ? S.box_lo_w[0] : S.box_lo[0]) - NEAR_GROW + cx;
        y = (pery ? S.box_lo_w[1] : S.box_lo[1]) - NEAR_GROW + cy;
        if (perx) { x += (x < 0) ? g.nx : 0; x -= (x >= g.nx) ? g.nx : 0; } else if (x < 0 || x >= g.nx) return;
        if (pery) { y += (y < 0) ? g.ny : 0; y -= (y >= g.ny) ? g.ny : 0; } else if (y < 0 || y >= g.ny) return;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            int zl = (perz ? S.box_lo_w[2] : S.box_lo[2]) - NEAR_GROW + cz + l;
            on[l] = cz + l < box.Bz + 2 * NEAR_GROW;
            if (perz) { zl += (zl < 0) ? g.nz : 0; zl -= (zl >= g.nz) ? g.nz : 0; }
            else on[l] = on[l] && zl >= 0 && zl < g.nz;
            z[l] = on[l] ? zl : 0;
        }
    } else {
        x = cx;
        y = cy;
        if (x >= g.nx || y >= g.ny) return;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            on[l] = cz + l < g.nz;
            z[l] = on[l] ? cz + l : 0;
        }
        if (MODE == K1_FAR) {
            // the z tests first: the planes are the same for a whole block
            bool xy_checked = false, in_xy = false;
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const int rz = rel_axis(z[l], S.box_lo[2], S.box_lo_w[2], NEAR_GROW, g.nz, perz);
                if (on[l] && (unsigned)rz < (unsigned)(box.Bz + 2 * NEAR_GROW)) {
                    if (!xy_checked) {
                        const int rx = rel_axis(x, S.box_lo[0], S.box_lo_w[0], NEAR_GROW, g.nx, perx);
                        const int ry = rel_axis(y, S.box_lo[1], S.box_lo_w[1], NEAR_GROW, g.ny, pery);
                        in_xy = (unsigned)rx < (unsigned)(box.Bx + 2 * NEAR_GROW) &&
                                (unsigned)ry < (unsigned)(box.By + 2 * NEAR_GROW);
                        xy_checked = true;
                    }
                    if (in_xy) on[l] = false;
                }
            }
        }
    }
    if (!on[0] && !on[1]) return;
    // a missing cell shares its partner's plane (loads in bounds, no store)
    if (!on[0]) z[0] = z[1];
    if (!on[1]) z[1] = z[0];
    f2 q[27];
    pull27x2<ST>(g, src, x, y, z[0], z[1], S.ring, S.reseed, utop_in, q);
    k1_pair_collide_store<ST, MODE>(g, dst, utop_out, S, hbox, box, x, y, z, on, q);
}

// The part of K1 after the pull, for a pair of cells (x, y, z[0]), (x, y,
// z[1]) whose pre-collision values are q (shared by the plain pull above and
// the staged kernels, so both run identical arithmetic).  STORE false: leave
// the post-collision values in q (storage domain) for the caller to store.
template <int ST, int MODE, bool STORE>
__device__ __forceinline__ void k1_pair_collide_store(const Geom &g, typename Codec<ST>::T *__restrict__ dst,
                                                      float *__restrict__ utop_out, const BodySlot &S,
                                                      const float *__restrict__ hbox, const BoxGeom &box, int x,
                                                      int y, const int z[2], const bool on[2], f2 q[27]) {
    const bool perx = g.bc_x == BC_PERIODIC, pery = g.bc_y == BC_PERIODIC, perz = g.bc_bottom == BC_PERIODIC;
    const int ring = S.ring;
    const f2 omega = make_float2(omega_of(g, z[0]), omega_of(g, z[1]));
    bool forced[2] = {false, false};
    f2 h[3] = {F2(0.0f), F2(0.0f), F2(0.0f)};
    f2 tau = F2(1.0f);
    if (MODE == K1_ALLF || MODE == K1_NEAR) {
        const int rx = rel_axis(x, S.box_lo[0], S.box_lo_w[0], 0, g.nx, perx);
        const int ry = rel_axis(y, S.box_lo[1], S.box_lo_w[1], 0, g.ny, pery);
        if ((unsigned)rx < (unsigned)box.Bx && (unsigned)ry < (unsigned)box.By) {
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const int rz = rel_axis(z[l], S.box_lo[2], S.box_lo_w[2], 0, g.nz, perz);
                if (on[l] && (unsigned)rz < (unsigned)box.Bz) {
                    const size_t b = ((size_t)rz * box.By + ry) * box.Bx + rx;
                    const float h0 = __ldg(hbox + b), h1 = __ldg(hbox + box.nbox + b), h2 = __ldg(hbox + 2 * box.nbox + b);
                    if (l == 0) { h[0].x = h0; h[1].x = h1; h[2].x = h2; }
                    else { h[0].y = h0; h[1].y = h1; h[2].y = h2; }
                    forced[l] = true;
                }
            }
        }
        tau = make_float2(tau_of(g, z[0]), tau_of(g, z[1]));
    }
    const Macro2 M = macro_of2(moments27x2<ST>(q));
#pragma unroll
    for (int l = 0; l < 2; ++l)
        if (on[l] && z[l] == g.nz - 1) {
            const size_t c = (size_t)y * g.nx + x;
            utop_out[c] = l ? M.ux.y : M.ux.x;
            utop_out[g.plane + c] = l ? M.uy.y : M.uy.x;
            utop_out[2 * g.plane + c] = l ? M.uz.y : M.uz.x;
        }
    collide_pair<ST>(M, omega, tau, forced[0] || forced[1], forced[0], forced[1], h,
                     (MODE == K1_ALLF || MODE == K1_NEAR) ? g.force_scheme : 0, q);
    if (!STORE) return;  // the caller stores q itself
    const int ncell = (int)g.ncell;
    const int oa = zphys(z[0], ring, g.nz) * (int)g.plane, ob = zphys(z[1], ring, g.nz) * (int)g.plane;
    typename Codec<ST>::T *d = dst + (y * g.nx + x);
    if (ST == ST_BF16 && g.sround) {
        // one hash per population serves both cells (its low and high halves)
        const int own = oa + y * g.nx + x;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const unsigned r = pcg_hash(sr_key(i * ncell + own, S.step));
            if (on[0]) store_bf16_sr(reinterpret_cast<__nv_bfloat16 *>(d + (i * ncell + oa)), q[i].x, r & 0xffffu);
            if (on[1]) store_bf16_sr(reinterpret_cast<__nv_bfloat16 *>(d + (i * ncell + ob)), q[i].y, r >> 16);
        }
        return;
    }
    if (on[0] && on[1]) {
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            Codec<ST>::store(d + (i * ncell + oa), q[i].x);
            Codec<ST>::store(d + (i * ncell + ob), q[i].y);
        }
    } else if (on[0]) {
#pragma unroll
        for (int i = 0; i < 27; ++i) Codec<ST>::store(d + (i * ncell + oa), q[i].x);
    } else {
#pragma unroll
        for (int i = 0; i < 27; ++i) Codec<ST>::store(d + (i * ncell + ob), q[i].y);
    }
}

// Tile of a 1-D block of blockDim.x threads over (x, y): tx threads along x,
// blockDim.x / tx rows along y, one plane (pz = 1) or pair of planes (pz = 2);
// block b of a region ex x ey x ez (ceil(ez / pz) plane groups), x fastest.
// cz is the first plane.
__device__ __forceinline__ void tile_coords(int b, int tx, int ex, int ey, int pz, int &cx, int &cy, int &cz) {
    const int ty = blockDim.x / tx;
    const int gx = (ex + tx - 1) / tx, gy = (ey + ty - 1) / ty;
    const int bx = b % gx, rest = b / gx;
    cx = bx * tx + (int)threadIdx.x % tx;
    cy = (rest % gy) * ty + (int)threadIdx.x / tx;
    cz = pz * (rest / gy);
}

}  // namespace turret
