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
    Macro M;
    M.drho = drho ? (float)drho[c] : 0.0f;
    M.rho = (float)(1.0 + (drho ? drho[c] : 0.0));
    M.ux = u ? (float)u[3 * c] : 0.0f;
    M.uy = u ? (float)u[3 * c + 1] : 0.0f;
    M.uz = u ? (float)u[3 * c + 2] : 0.0f;
    M.Pxx = M.Pyy = M.Pzz = M.Pxy = M.Pxz = M.Pyz = 0.0f;
    float q[27];
    collide_factored<ST>(M, 1.0f, 1.0f, false, 0.0f, 0.0f, 0.0f, 0, q);
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
    const Macro M = macro_of(moments27<ST>(q));
    out[c] = M.rho;
    out[g.ncell + c] = M.ux;
    out[2 * g.ncell + c] = M.uy;
    out[3 * g.ncell + c] = M.uz;
}

template <int ST>
__global__ void __launch_bounds__(MB_THREADS) k_box_moments_bin(Geom g, const typename Codec<ST>::T *__restrict__ src,
                                                                const float *__restrict__ utop_in,
                                                                const DevState *__restrict__ st, int slot, BoxGeom box,
                                                                BoxArrays ba, int nmom, int nm,
                                                                const int *__restrict__ mbase,
                                                                const int *__restrict__ mseg,
                                                                int *__restrict__ tile_list,
                                                                int *__restrict__ tile_count, int cap, DevState *stw,
                                                                float rmin, float rmax) {
    mb_block<ST>(g, src, utop_in, st, slot, box, ba, nmom, nm, mbase, mseg, tile_list, tile_count, cap, stw, rmin, rmax,
                 blockIdx.x);
}

// ---------------------------------------------------------------------------
// Launchers.
static dim3 cell_grid(const Geom &g) { return dim3((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz); }
// collide+stream over the window: one thread per pair of planes
static dim3 pair_grid(const Geom &g) { return dim3((g.nx + 31) / 32, (g.ny + 3) / 4, (g.nz + 1) / 2); }
static dim3 near_grid(const BoxGeom &b) {
    const int ex = b.Bx + 2 * NEAR_MARGIN, ey = b.By + 2 * NEAR_MARGIN, ez = b.Bz + 2 * NEAR_MARGIN;
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

// Plan of a re-injection from the body slot: the copied planes [z0, z1) and
// the jump dz (false: no re-injection this step).  Every thread of the three
// kernels derives the same plan from the same slot (the origin changes last).
__device__ __forceinline__ bool reinject_plan(const Geom &g, const BodySlot &S, const Reinject &rj, int &z0, int &z1,
                                              int &dz) {
    const double zc = S.r[2] - (double)S.origin[2];
    if (!(zc < (double)rj.trigger)) return false;
    const int zf = (int)floor(zc);
    dz = rj.target - zf;
    if (dz <= 0) return false;
    z0 = max(zf - rj.below, 0);
    z1 = min(zf + rj.above, g.nz - dz);
    return true;
}

// pass 0: stage[i][z] = buf[i][z]; pass 1: buf[i][z + dz] = stage[i][z], for
// z in [z0, z1) and every population and cell of a plane (grid-stride: the
// launch is small, and nearly free on the steps without a re-injection)
template <typename T>
__global__ void k_reinject_copy(Geom g, T *__restrict__ buf, T *__restrict__ stage, const DevState *st, int slot,
                                Reinject rj, int pass) {
    int z0, z1, dz;
    if (!reinject_plan(g, st->s[slot], rj, z0, z1, dz) || z1 <= z0) return;
    const long long per_pop = (long long)(z1 - z0) * g.plane;
    const long long total = 27 * per_pop;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = k / per_pop, r = k - i * per_pop;
        const size_t from = (size_t)i * g.ncell + (size_t)z0 * g.plane + r;
        if (pass == 0) stage[from] = buf[from];
        else buf[from + (size_t)dz * g.plane] = stage[from];
    }
}

__global__ void k_reinject_origin(Geom g, DevState *st, int slot, Reinject rj) {
    int z0, z1, dz;
    if (threadIdx.x == 0 && reinject_plan(g, st->s[slot], rj, z0, z1, dz)) {
        BodySlot &S = st->s[slot];
        S.origin[2] -= dz;
        S.Ci[2] += dz;
        S.box_lo[2] += dz;
        S.box_lo_w[2] += dz;
    }
}

template <typename T>
static cudaError_t reinject_t(const Geom &g, void *buf, void *stage, DevState *st, int slot, const Reinject &rj,
                              cudaStream_t s) {
    if (rj.below + rj.above > 0) {
        k_reinject_copy<T><<<608, 256, 0, s>>>(g, (T *)buf, (T *)stage, st, slot, rj, 0);
        k_reinject_copy<T><<<608, 256, 0, s>>>(g, (T *)buf, (T *)stage, st, slot, rj, 1);
    }
    k_reinject_origin<<<1, 32, 0, s>>>(g, st, slot, rj);
    return cudaGetLastError();
}

cudaError_t launch_reinject(const Geom &g, int storage, void *buf, void *stage, DevState *st, int slot,
                            const Reinject &rj, cudaStream_t s) {
    return storage == ST_F32 ? reinject_t<float>(g, buf, stage, st, slot, rj, s)
                             : reinject_t<unsigned short>(g, buf, stage, st, slot, rj, s);
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

cudaError_t launch_box_moments_bin(const Geom &g, int storage, const void *src, const float *utop_in,
                                   const DevState *st, int slot, const BoxGeom &box, BoxArrays ba, int nm,
                                   const int *mbase, const int *mseg, int *tile_list, int *tile_count, int cap,
                                   DevState *stw, float rmin, float rmax, cudaStream_t s) {
    const int nmom = (int)((box.nbox + MB_THREADS - 1) / MB_THREADS);
    const unsigned nb = (unsigned)(nmom + box.tx * box.ty * box.tz);
    switch (storage) {
        case ST_F32: k_box_moments_bin<ST_F32><<<nb, MB_THREADS, 0, s>>>(g, (const float *)src, utop_in, st, slot, box, ba, nmom, nm, mbase, mseg, tile_list, tile_count, cap, stw, rmin, rmax); break;
        case ST_F16: k_box_moments_bin<ST_F16><<<nb, MB_THREADS, 0, s>>>(g, (const __half *)src, utop_in, st, slot, box, ba, nmom, nm, mbase, mseg, tile_list, tile_count, cap, stw, rmin, rmax); break;
        default: k_box_moments_bin<ST_BF16><<<nb, MB_THREADS, 0, s>>>(g, (const __nv_bfloat16 *)src, utop_in, st, slot, box, ba, nmom, nm, mbase, mseg, tile_list, tile_count, cap, stw, rmin, rmax); break;
    }
    return cudaGetLastError();
}

}  // namespace turret
