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
//   rebuild : per-axis factors X, X', X'' and five terms per (y, z) pair that
//             carry the equilibrium and the off-equilibrium parts together,
//             then 3 FMAs per population (collide_rr below)
// about 335 FP32 operations per cell.  Populations are stored as deviations
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
// RXS-M-XS output permutation -- applied to a key made of a stored element's
// index and the time step, so a run is reproducible bit for bit.  One hash
// serves the two elements 2k and 2k + 1 of a population array (x-adjacent
// cells when nx is even): the low 16 bits the even one, the high 16 the odd
// one, so every kernel gives an element the same bits however it pairs cells.
__device__ __forceinline__ unsigned pcg_hash(unsigned v) {
    const unsigned state = v * 747796405u + 2891336453u;
    const unsigned word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}
__device__ __forceinline__ unsigned sr_key(int element, long long step) {
    return (unsigned)element + 0x9E3779B9u * (unsigned)step;
}
// The 16 random bits of element e (its index in the population arrays).
__device__ __forceinline__ unsigned sr_bits(int e, long long step) {
    const unsigned h = pcg_hash(sr_key(e & ~1, step));
    return (e & 1) ? h >> 16 : h & 0xffffu;
}
// bf16 bits of r with its magnitude rounded up with probability equal to the
// dropped fraction of the last kept bit (16 random bits added below the kept
// bits, then truncated): unbiased, E[stored] = r.
__device__ __forceinline__ unsigned short bf16_sr_bits(float r, unsigned rnd16) {
    return (unsigned short)((__float_as_uint(r) + rnd16) >> 16);
}
__device__ __forceinline__ void store_bf16_sr(__nv_bfloat16 *p, float r, unsigned rnd16) {
    *reinterpret_cast<unsigned short *>(p) = bf16_sr_bits(r, rnd16);
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

// ---------------------------------------------------------------------------
// Lane-generic arithmetic of the moments and the collision: V = float (one
// cell) or f2 (two cells, one packed f32x2 instruction per operation).  Every
// operation is a hand-written add/sub/mul/fma.rn instruction (.f32 or
// .f32x2), which the compiler keeps as written: with explicit rounding it
// fuses nothing.  (The packed intrinsics of CUDA 13.0 were measured to fuse a
// multiply whose only use is an add into one FMA, even under -fmad=false, so
// the scalar and packed forms of the same source rounded differently.)  A
// packed instruction rounds each lane as the scalar one does, so a cell gets
// the same bits whichever form computes it and whatever cell it is paired with.
typedef float2 f2;
__device__ __forceinline__ f2 F2(float a) { return make_float2(a, a); }

__device__ __forceinline__ float vadd(float a, float b) {
    float r;
    asm("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float vsub(float a, float b) {
    float r;
    asm("sub.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float vmul(float a, float b) {
    float r;
    asm("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float vfma(float a, float b, float c) {
    float r;
    asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float vrcp(float a) { return __frcp_rn(a); }
__device__ __forceinline__ unsigned long long f2_u64(f2 a) {
    return (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
}
__device__ __forceinline__ f2 u64_f2(unsigned long long a) {
    return make_float2(__uint_as_float((unsigned)a), __uint_as_float((unsigned)(a >> 32)));
}
__device__ __forceinline__ f2 vadd(f2 a, f2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_u64(a)), "l"(f2_u64(b)));
    return u64_f2(r);
}
__device__ __forceinline__ f2 vsub(f2 a, f2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_u64(a)), "l"(f2_u64(b)));
    return u64_f2(r);
}
__device__ __forceinline__ f2 vmul(f2 a, f2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_u64(a)), "l"(f2_u64(b)));
    return u64_f2(r);
}
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_u64(a)), "l"(f2_u64(b)), "l"(f2_u64(c)));
    return u64_f2(r);
}
__device__ __forceinline__ f2 vrcp(f2 a) { return make_float2(__frcp_rn(a.x), __frcp_rn(a.y)); }
template <class V>
__device__ __forceinline__ V vs(float a);
template <>
__device__ __forceinline__ float vs<float>(float a) { return a; }
template <>
__device__ __forceinline__ f2 vs<f2>(float a) { return F2(a); }
// a times a power of two c (exact; no operation for c = 1)
template <class V>
__device__ __forceinline__ V vpow2(V a, float c) { return c == 1.0f ? a : vmul(a, vs<V>(c)); }

// Raw moments of the stored values up to second order, by three separable
// 3-point passes: drho = sum r, the momentum negated (nj = -sum xi r, which
// costs nothing here and keeps the stress below free of a multiply feeding an
// add) and Pi'_ab = sum xi_a xi_b r.  FP32 storage holds r_i = s_i = 216 (f_i
// - w_i); the 16-bit domains r_i = K s_i / W_i carry the axis weights W1 = (1,
// 4, 1) in the sums that need them (the 4 sits on xi = 0, where the
// xi-weighted sums vanish anyway).  Every moment here is thus K times the
// scaled moment, which is 216 times the physical one (K = 1 for FP32 and BF16).
template <class V>
struct MomR {
    V drho, njx, njy, njz, pxx, pyy, pzz, pxy, pxz, pyz;
};

// a + W1(1) b + c in the storage domain
template <bool SC, class V>
__device__ __forceinline__ V wsum3(V a, V b, V c) {
    return SC ? vfma(vs<V>(4.0f), b, vadd(a, c)) : vadd(vadd(a, b), c);
}

template <int ST, class V>
__device__ __forceinline__ MomR<V> moments_raw(const V q[27]) {
    constexpr bool SC = Codec<ST>::scaled;
    V A0[9], A1[9], A2[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {  // x pass, k = ey + 3 ez
        const V a = q[3 * k], b = q[3 * k + 1], c = q[3 * k + 2];
        A0[k] = wsum3<SC>(a, b, c);
        A1[k] = vsub(a, c);  // -sum xi_x r
        A2[k] = vadd(c, a);
    }
    V B00[3], B01[3], B02[3], B10[3], B11[3], B20[3];
#pragma unroll
    for (int ez = 0; ez < 3; ++ez) {  // y pass
        const int k = 3 * ez;
        B00[ez] = wsum3<SC>(A0[k], A0[k + 1], A0[k + 2]);
        B01[ez] = vsub(A0[k], A0[k + 2]);  // -sum xi_y
        B02[ez] = vadd(A0[k + 2], A0[k]);
        B10[ez] = wsum3<SC>(A1[k], A1[k + 1], A1[k + 2]);
        B11[ez] = vsub(A1[k], A1[k + 2]);  // +sum xi_x xi_y
        B20[ez] = wsum3<SC>(A2[k], A2[k + 1], A2[k + 2]);
    }
    MomR<V> m;  // z pass
    m.drho = wsum3<SC>(B00[0], B00[1], B00[2]);
    m.njz = vsub(B00[0], B00[2]);
    m.pzz = vadd(B00[2], B00[0]);
    m.njy = wsum3<SC>(B01[0], B01[1], B01[2]);
    m.pyz = vsub(B01[0], B01[2]);
    m.pyy = wsum3<SC>(B02[0], B02[1], B02[2]);
    m.njx = wsum3<SC>(B10[0], B10[1], B10[2]);
    m.pxz = vsub(B10[0], B10[2]);
    m.pxy = wsum3<SC>(B11[0], B11[1], B11[2]);
    m.pxx = wsum3<SC>(B20[0], B20[1], B20[2]);
    return m;
}

// Macroscopic quantities from the raw moments (tilde: 216 times physical):
//   drho = drho~ / 216, rho = 1 + drho, u = j~ / (216 + drho~),
//   P_ab = K P1~_ab,  P1~ = Pi'~ - drho~ I / 3 - j~ u^T  (= 216 [Pi - rho (I/3 + u u)]).
// K is a power of two, so taking the raw sums without dividing them by K
// changes no bit of drho or u (216 K + K drho~ and K j~ round as the unscaled
// sums, scaled); u = (-j)(-1 / (216 K + drho)) has the bits of j / (...).
// Each stress component is one or two FMAs, so it is rounded once or twice.
template <class V>
struct MacroR {
    V drho, rho, ux, uy, uz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz;
};

template <int ST, class V>
__device__ __forceinline__ MacroR<V> macro_raw(const MomR<V> &m) {
    constexpr float K = Codec<ST>::K;
    MacroR<V> M;
    M.drho = vmul(m.drho, vs<V>(INV_SCALE / K));
    M.rho = vfma(m.drho, vs<V>(INV_SCALE / K), vs<V>(1.0f));
    const V nir = vrcp(vsub(vs<V>(-SCALE * K), m.drho));
    M.ux = vmul(m.njx, nir);
    M.uy = vmul(m.njy, nir);
    M.uz = vmul(m.njz, nir);
    M.Pxx = vfma(m.njx, M.ux, vfma(m.drho, vs<V>(-1.0f / 3.0f), m.pxx));
    M.Pyy = vfma(m.njy, M.uy, vfma(m.drho, vs<V>(-1.0f / 3.0f), m.pyy));
    M.Pzz = vfma(m.njz, M.uz, vfma(m.drho, vs<V>(-1.0f / 3.0f), m.pzz));
    M.Pxy = vfma(m.njx, M.uy, m.pxy);
    M.Pxz = vfma(m.njx, M.uz, m.pxz);
    M.Pyz = vfma(m.njy, M.uz, m.pyz);
    return M;
}

// Per-axis factors of the collision.  With m(u) = prod_a u_a^{p_a} and the
// weighted basis g_p(xi) = w1(xi) H_p(xi), every term of the post-collision
// Hermite expansion is an outer product of one 3-vector per axis, so each
// population is rebuilt directly from per-axis vectors (here scaled by 6 so
// that the weights 6 w1 = W1 = (1, 4, 1) are exact):
//   X(e)   = 6 sum_p u^p g_p(e)      = W1(e) (1 + a(e)),  a = (-3u+3u^2, -3u^2/2, 3u+3u^2)
//   X'(e)  = 6 sum_p p u^(p-1) g_p(e) = (6u - 3, -12u, 6u + 3)
//   X''(e) = 6 sum_p p(p-1) u^(p-2) g_p(e) = (6, -12, 6).
// In the scaled storage domains every factor is divided by W1(e), which
// divides each product by W_i: X / W1 = 1 + a, X' / W1, X'' / W1 = (6, -3, 6).
template <class V>
struct AxisR {
    V a[3], X[3], Xp[3];
};

template <bool SC, class V>
__device__ __forceinline__ AxisR<V> axis_r(V u) {
    AxisR<V> f;
    const V u2 = vmul(u, u), tm = vfma(u, u, vmul(u, vs<V>(-1.0f))), tp = vfma(u, u, u);  // u^2 -+ u
    f.a[0] = vmul(vs<V>(3.0f), tm);
    f.a[1] = vmul(vs<V>(-1.5f), u2);
    f.a[2] = vmul(vs<V>(3.0f), tp);
    f.X[0] = vfma(vs<V>(3.0f), tm, vs<V>(1.0f));
    f.X[1] = SC ? vfma(vs<V>(-1.5f), u2, vs<V>(1.0f)) : vmul(vs<V>(4.0f), vfma(vs<V>(-1.5f), u2, vs<V>(1.0f)));
    f.X[2] = vfma(vs<V>(3.0f), tp, vs<V>(1.0f));
    f.Xp[0] = vfma(vs<V>(6.0f), u, vs<V>(-3.0f));
    f.Xp[1] = vmul(vs<V>(SC ? -3.0f : -12.0f), u);
    f.Xp[2] = vfma(vs<V>(6.0f), u, vs<V>(3.0f));
    return f;
}

// Post-collision values in the storage domain of ST (FP32: s_i = 216 (f*_i -
// w_i); 16-bit: K s_i / W_i) from the macroscopic state, as f* = f0 + (1 -
// 1/tau) f1 (Eq. 7) with f1 rebuilt from P1 (Eq. A.3).  With Y, Z the factors
// X of the y and z axes, W = W1 in the storage domain (1 in the 16-bit ones),
// Aw = W a, r = K rho, d = K drho and P' = (1 - 1/tau) P1:
//   G0 = P'xx/2 Y Z,  G1 = P'yy/2 Y'' Z + P'zz/2 Y Z'' + P'yz Y' Z',
//   G2 = P'xy Y' Z + P'xz Y Z'                  (off-equilibrium, per (y, z));
// the equilibrium deviation W_i (r E + d), E = (1+a_x)(1+a_y)(1+a_z) - 1,
// splits as Aw_x G3 + W_x G4 with G3 = r Y Z and G4 = r Aw_y Z + W_y W_z
// (r a_z + d); and X_x = W_x + Aw_x.  So every value is three FMAs from five
// per-(y, z) terms,
//   s_i = X''_x G0 + Aw_x (G1 + G3) + X'_x G2 + W_x (G1 + G4),
// with no O(1) term cancelling (G3 enters only multiplied by a_x).
// Forced lanes take the equilibrium c1 f0(u) + c2 f0(v), v = u + tau h
// (Eq. 15 reading: scheme 0 c = (1 - omega, omega), scheme 1 (0, 1)); the
// unforced lanes of a forced pair pass c = (1, 0) and h = 0 and get the values
// of the unforced form (an exact zero may come out with the other sign).
template <int ST, class V>
__device__ __forceinline__ void collide_rr(const MacroR<V> &M, V omega, bool anyforced, V c1, V c2, V tau,
                                           const V h[3], V s[27]) {
    constexpr bool SC = Codec<ST>::scaled;
    constexpr float K = Codec<ST>::K;
    const float xpp[3] = {6.0f, SC ? -3.0f : -12.0f, 6.0f};  // X''
    const float w[3] = {1.0f, SC ? 1.0f : 4.0f, 1.0f};        // W1 in the storage domain
    const AxisR<V> fx = axis_r<SC>(M.ux), fy = axis_r<SC>(M.uy), fz = axis_r<SC>(M.uz);
    // P' (storage domain) = (1 - omega) P / 216: hxx = P'xx / 2, pxy = P'xy, ...
    const V o1 = vmul(vsub(vs<V>(1.0f), omega), vs<V>(INV_SCALE));
    const V oh = vmul(o1, vs<V>(0.5f));
    const V hxx = vmul(oh, M.Pxx), hyy = vmul(oh, M.Pyy), hzz = vmul(oh, M.Pzz);
    const V pxy = vmul(o1, M.Pxy), pxz = vmul(o1, M.Pxz), pyz = vmul(o1, M.Pyz);
    V cY[3], cZ[3], bY[3], aY[3], bZ[3], HZ[3], Ax[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        cY[e] = vmul(hyy, vs<V>(xpp[e]));  // P'yy/2 Y''
        cZ[e] = vmul(hzz, vs<V>(xpp[e]));  // P'zz/2 Z''
        bY[e] = vmul(pyz, fy.Xp[e]);       // P'yz Y'
        aY[e] = vmul(pxy, fy.Xp[e]);       // P'xy Y'
        bZ[e] = vmul(pxz, fz.Xp[e]);       // P'xz Z'
        HZ[e] = vmul(hxx, fz.X[e]);        // P'xx/2 Z
        Ax[e] = vpow2(fx.a[e], w[e]);      // Aw_x
    }
    const V r = vpow2(M.rho, K), d = vpow2(M.drho, K);
    if (!anyforced) {
        V rY[3], rA[3], Qz[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            rY[e] = vmul(r, fy.X[e]);
            rA[e] = vpow2(vmul(r, fy.a[e]), w[e]);
            Qz[e] = vpow2(vfma(r, fz.a[e], d), w[e]);
        }
#pragma unroll
        for (int ez = 0; ez < 3; ++ez)
#pragma unroll
            for (int ey = 0; ey < 3; ++ey) {
                const V Y = fy.X[ey], Z = fz.X[ez];
                const V G0 = vmul(Y, HZ[ez]);
                const V G1 = vfma(cY[ey], Z, vfma(Y, cZ[ez], vmul(bY[ey], fz.Xp[ez])));
                const V G2 = vfma(aY[ey], Z, vmul(Y, bZ[ez]));
                const V G4 = vfma(rA[ey], Z, vpow2(Qz[ez], w[ey]));
                const V G13 = vfma(rY[ey], Z, G1), G14 = vadd(G1, G4);  // G1 + G3, G1 + G4
#pragma unroll
                for (int ex = 0; ex < 3; ++ex)
                    s[ex + 3 * ey + 9 * ez] =
                        vfma(vs<V>(xpp[ex]), G0, vfma(Ax[ex], G13, vfma(fx.Xp[ex], G2, vpow2(G14, w[ex]))));
            }
        return;
    }
    const AxisR<V> gx = axis_r<SC>(vfma(tau, h[0], M.ux)), gy = axis_r<SC>(vfma(tau, h[1], M.uy)),
                   gz = axis_r<SC>(vfma(tau, h[2], M.uz));
    const V r1 = vmul(c1, r), d1 = vmul(c1, d), r2 = vmul(c2, r), d2 = vmul(c2, d);
    V rY1[3], rA1[3], Qz1[3], rY2[3], rA2[3], Qz2[3], Bx[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        rY1[e] = vmul(r1, fy.X[e]);
        rA1[e] = vpow2(vmul(r1, fy.a[e]), w[e]);
        Qz1[e] = vpow2(vfma(r1, fz.a[e], d1), w[e]);
        rY2[e] = vmul(r2, gy.X[e]);
        rA2[e] = vpow2(vmul(r2, gy.a[e]), w[e]);
        Qz2[e] = vpow2(vfma(r2, gz.a[e], d2), w[e]);
        Bx[e] = vpow2(gx.a[e], w[e]);
    }
#pragma unroll
    for (int ez = 0; ez < 3; ++ez)
#pragma unroll
        for (int ey = 0; ey < 3; ++ey) {
            const V Y = fy.X[ey], Z = fz.X[ez];
            const V G0 = vmul(Y, HZ[ez]);
            const V G1 = vfma(cY[ey], Z, vfma(Y, cZ[ez], vmul(bY[ey], fz.Xp[ez])));
            const V G2 = vfma(aY[ey], Z, vmul(Y, bZ[ez]));
            const V G3v = vmul(rY2[ey], gz.X[ez]);
            const V G4 = vadd(vfma(rA1[ey], Z, vpow2(Qz1[ez], w[ey])), vfma(rA2[ey], gz.X[ez], vpow2(Qz2[ez], w[ey])));
            const V G13 = vfma(rY1[ey], Z, G1), G14 = vadd(G1, G4);
#pragma unroll
            for (int ex = 0; ex < 3; ++ex)
                s[ex + 3 * ey + 9 * ez] = vfma(vs<V>(xpp[ex]), G0,
                                               vfma(Ax[ex], G13, vfma(Bx[ex], G3v, vfma(fx.Xp[ex], G2, vpow2(G14, w[ex])))));
        }
}

// Equilibrium weights of a lane (see collide_rr): unforced (1, 0); forced
// scheme 0 (1 - omega, omega), scheme 1 (0, 1).
__device__ __forceinline__ void forcing_weights(float omega, bool forced, int scheme, float &c1, float &c2) {
    c1 = !forced ? 1.0f : (scheme == 1 ? 0.0f : 1.0f - omega);
    c2 = !forced ? 0.0f : (scheme == 1 ? 1.0f : omega);
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
    const MacroR<float> M = macro_raw<ST>(moments_raw<ST>(q));
    if (zl == g.nz - 1) {
        const size_t c = (size_t)y * g.nx + x;
        utop_out[c] = M.ux;
        utop_out[g.plane + c] = M.uy;
        utop_out[2 * g.plane + c] = M.uz;
    }
    float c1, c2;
    forcing_weights(omega, forced, g.force_scheme, c1, c2);
    const float h[3] = {hx, hy, hz};
    const float tau = (MODE == K1_ALLF || MODE == K1_NEAR) ? tau_of(g, zl) : 1.0f;
    collide_rr<ST>(M, omega, forced, c1, c2, tau, h, q);
    const int oz = zphys(zl, ring, g.nz) * (int)g.plane;
    const int ncell = (int)g.ncell;
    typename Codec<ST>::T *d = dst + (y * g.nx + x);
    if (ST == ST_BF16 && g.sround) {
        const int own = oz + y * g.nx + x;
#pragma unroll
        for (int i = 0; i < 27; ++i)
            store_bf16_sr(reinterpret_cast<__nv_bfloat16 *>(d + (i * ncell + oz)), q[i], sr_bits(i * ncell + own, S.step));
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
    const MacroR<f2> M = macro_raw<ST>(moments_raw<ST>(q));
#pragma unroll
    for (int l = 0; l < 2; ++l)
        if (on[l] && z[l] == g.nz - 1) {
            const size_t c = (size_t)y * g.nx + x;
            utop_out[c] = l ? M.ux.y : M.ux.x;
            utop_out[g.plane + c] = l ? M.uy.y : M.uy.x;
            utop_out[2 * g.plane + c] = l ? M.uz.y : M.uz.x;
        }
    f2 c1, c2;
    forcing_weights(omega.x, forced[0], g.force_scheme, c1.x, c2.x);
    forcing_weights(omega.y, forced[1], g.force_scheme, c1.y, c2.y);
    collide_rr<ST>(M, omega, forced[0] || forced[1], c1, c2, tau, h, q);
    if (!STORE) return;  // the caller stores q itself
    const int ncell = (int)g.ncell;
    const int oa = zphys(z[0], ring, g.nz) * (int)g.plane, ob = zphys(z[1], ring, g.nz) * (int)g.plane;
    typename Codec<ST>::T *d = dst + (y * g.nx + x);
    if (ST == ST_BF16 && g.sround) {
        const int own_a = oa + y * g.nx + x, own_b = ob + y * g.nx + x;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            if (on[0])
                store_bf16_sr(reinterpret_cast<__nv_bfloat16 *>(d + (i * ncell + oa)), q[i].x, sr_bits(i * ncell + own_a, S.step));
            if (on[1])
                store_bf16_sr(reinterpret_cast<__nv_bfloat16 *>(d + (i * ncell + ob)), q[i].y, sr_bits(i * ncell + own_b, S.step));
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
