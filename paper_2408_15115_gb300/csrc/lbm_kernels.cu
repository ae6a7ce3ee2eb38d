// lbm_kernels.cu -- single-run kernels of the fused collide+stream and of the
// passes sharing its streaming and moment code (cell code in lbm_cell.cuh).
#include "lbm_cell.cuh"

namespace turret {

// Window launches with 16-bit storage: five blocks per SM (<= 102 registers, a
// few spilled values in L1) measured faster than four; FP32 keeps four (128
// registers, no spill); the small near-region launch is left unconstrained.
template <int ST, int MODE>
__global__ void __launch_bounds__(128, MODE == K1_NEAR ? 1 : (ST == ST_F32 ? 4 : 5)) k_collide_stream(Geom g, const typename Codec<ST>::T *__restrict__ src,
                                                        typename Codec<ST>::T *__restrict__ dst,
                                                        const float *__restrict__ utop_in,
                                                        float *__restrict__ utop_out, DevState *st, int slot,
                                                        int slot_out, const float *__restrict__ hbox, BoxGeom box) {
    if (slot_out >= 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
        threadIdx.y == 0) {
        // carry the body and window to the next time level (no entering plane there)
        st->s[slot_out] = st->s[slot];
        st->s[slot_out].reseed = -1;
        st->s[slot_out].step += 1;
    }
    if (MODE == K1_NEAR)  // small, on the critical path: one cell per thread
        k1_cell<ST, MODE>(g, src, dst, utop_in, utop_out, st->s[slot], hbox, box, blockIdx.x * 32 + threadIdx.x,
                          blockIdx.y * 4 + threadIdx.y, blockIdx.z);
    else  // the window: a pair of planes per thread
        k1_pair<ST, MODE>(g, src, dst, utop_in, utop_out, st->s[slot], hbox, box, blockIdx.x * 32 + threadIdx.x,
                          blockIdx.y * 4 + threadIdx.y, 2 * blockIdx.z);
}


// Equilibrium of given (rho - 1, u) fields (doubles, window order) as the
// post-collision state; u of the top plane goes to the pressure-ghost buffer.
template <int ST>
__global__ void k_init_equilibrium(Geom g, typename Codec<ST>::T *__restrict__ dst, const double *__restrict__ drho,
                                   const double *__restrict__ u, float *__restrict__ utop) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    MacroR<float> M;
    M.drho = drho ? (float)drho[c] : 0.0f;
    M.rho = (float)(1.0 + (drho ? drho[c] : 0.0));
    M.ux = u ? (float)u[3 * c] : 0.0f;
    M.uy = u ? (float)u[3 * c + 1] : 0.0f;
    M.uz = u ? (float)u[3 * c + 2] : 0.0f;
    M.Pxx = M.Pyy = M.Pzz = M.Pxy = M.Pxz = M.Pyz = 0.0f;
    float q[27];
    const float h[3] = {0.0f, 0.0f, 0.0f};
    collide_rr<ST>(M, 1.0f, false, 1.0f, 0.0f, 1.0f, h, q);
#pragma unroll
    for (int i = 0; i < 27; ++i) Codec<ST>::store(dst + (size_t)i * g.ncell + c, q[i]);
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
                                               int slot, float *__restrict__ out, int pops) {
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 4 + threadIdx.y;
    const int zl = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    float q[27];
    pull27<ST>(g, src, x, y, zl, st->s[slot].ring, st->s[slot].reseed, utop_in, q);
    const size_t c = ((size_t)zl * g.ny + y) * g.nx + x;
    if (pops) {  // f_i - w_i = s_i / 216 = r_i W_i / (216 K)
#pragma unroll
        for (int i = 0; i < 27; ++i)
            out[(size_t)i * g.ncell + c] = q[i] * ((Codec<ST>::scaled ? Wq(i) / Codec<ST>::K : 1.0f) * INV_SCALE);
        return;
    }
    const MacroR<float> M = macro_raw<ST>(moments_raw<ST>(q));
    out[c] = M.rho;
    out[g.ncell + c] = M.ux;
    out[2 * g.ncell + c] = M.uy;
    out[3 * g.ncell + c] = M.uz;
}


// ---------------------------------------------------------------------------
// Launchers.
static dim3 cell_grid(const Geom &g) { return dim3((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz); }
// collide+stream over the window: one thread per pair of planes
static dim3 pair_grid(const Geom &g) { return dim3((g.nx + 31) / 32, (g.ny + 3) / 4, (g.nz + 1) / 2); }
static dim3 near_grid(const BoxGeom &b) {
    const int ex = b.Bx + 2 * NEAR_GROW, ey = b.By + 2 * NEAR_GROW, ez = b.Bz + 2 * NEAR_GROW;
    return dim3((ex + 31) / 32, (ey + 3) / 4, ez);
}

template <int ST>
static cudaError_t collide_t(const Geom &g, const void *src, void *dst, const float *utop_in, float *utop_out,
                             DevState *st, int slot, int slot_out, const float *hbox, const BoxGeom &box,
                             bool has_box, int region, cudaStream_t s) {
    using T = typename Codec<ST>::T;
    const dim3 blk(32, 4);
    const T *fs = (const T *)src;
    T *fd = (T *)dst;
    if (region == REGION_NEAR)
        k_collide_stream<ST, K1_NEAR><<<near_grid(box), blk, 0, s>>>(g, fs, fd, utop_in, utop_out, st, slot, slot_out, hbox, box);
    else if (region == REGION_FAR)
        k_collide_stream<ST, K1_FAR><<<pair_grid(g), blk, 0, s>>>(g, fs, fd, utop_in, utop_out, st, slot, slot_out, hbox, box);
    else if (has_box)
        k_collide_stream<ST, K1_ALLF><<<pair_grid(g), blk, 0, s>>>(g, fs, fd, utop_in, utop_out, st, slot, slot_out, hbox, box);
    else
        k_collide_stream<ST, K1_ALL><<<pair_grid(g), blk, 0, s>>>(g, fs, fd, utop_in, utop_out, st, slot, slot_out, hbox, box);
    return cudaGetLastError();
}

cudaError_t launch_collide_stream(const Geom &g, int storage, const void *src, void *dst, const float *utop_in,
                                  float *utop_out, DevState *st, int slot, int slot_out, const float *hbox,
                                  const BoxGeom &box, bool has_box, int region, cudaStream_t s) {
    switch (storage) {
        case ST_F32: return collide_t<ST_F32>(g, src, dst, utop_in, utop_out, st, slot, slot_out, hbox, box, has_box, region, s);
        case ST_F16: return collide_t<ST_F16>(g, src, dst, utop_in, utop_out, st, slot, slot_out, hbox, box, has_box, region, s);
        default: return collide_t<ST_BF16>(g, src, dst, utop_in, utop_out, st, slot, slot_out, hbox, box, has_box, region, s);
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
                         int slot, float *out, bool pops, cudaStream_t s) {
    switch (storage) {
        case ST_F32: k_macro<ST_F32><<<cell_grid(g), dim3(32, 4), 0, s>>>(g, (const float *)src, utop_in, st, slot, out, pops); break;
        case ST_F16: k_macro<ST_F16><<<cell_grid(g), dim3(32, 4), 0, s>>>(g, (const __half *)src, utop_in, st, slot, out, pops); break;
        default: k_macro<ST_BF16><<<cell_grid(g), dim3(32, 4), 0, s>>>(g, (const __nv_bfloat16 *)src, utop_in, st, slot, out, pops); break;
    }
    return cudaGetLastError();
}


}  // namespace turret
