// lbm_far.cu -- the far-cell collide+stream of a coupled single-run step with
// FP32 storage, under a register cap.
//
// In the step graph this launch shares the SMs with the immersed-boundary
// chain.  At 128 registers its four resident blocks of 128 threads fill the
// 65,536-register file, so any chain block resident on an SM displaces one of
// them (a quarter of that SM's streaming).  At 120 registers (no spill) four
// blocks leave 4,096 registers free, room for a small chain block (the
// 64-thread interpolation blocks) beside them.  The cell code is the same
// device function as every other collide+stream launch (lbm_cell.cuh), so
// results are identical.
#include "lbm_cell.cuh"

namespace turret {

__global__ void __maxnreg__(120) k_collide_stream_far_f32(Geom g, const float *__restrict__ src,
                                                          float *__restrict__ dst, const float *__restrict__ utop_in,
                                                          float *__restrict__ utop_out, DevState *st, int slot,
                                                          const float *__restrict__ hbox, BoxGeom box) {
    k1_pair<ST_F32, K1_FAR>(g, src, dst, utop_in, utop_out, st->s[slot], hbox, box, blockIdx.x * 32 + threadIdx.x,
                            blockIdx.y * 4 + threadIdx.y, 2 * blockIdx.z);
}

cudaError_t launch_collide_far(const Geom &g, int storage, const void *src, void *dst, const float *utop_in,
                               float *utop_out, DevState *st, int slot, const float *hbox, const BoxGeom &box,
                               cudaStream_t s, const CUtensorMap *lmap, const CUtensorMap *smap) {
    if (storage != ST_F32 && lmap && smap)
        return launch_collide_staged(g, storage, *lmap, *smap, src, dst, utop_in, utop_out, st, slot, -1, hbox, box,
                                     REGION_FAR, s);
    if (storage != ST_F32 && xpair_eligible(g, storage))
        return launch_collide_xpair(g, storage, src, dst, utop_in, utop_out, st, slot, -1, hbox, box, REGION_FAR, s);
    if (storage != ST_F32)
        return launch_collide_stream(g, storage, src, dst, utop_in, utop_out, st, slot, -1, hbox, box, true,
                                     REGION_FAR, s);
    const dim3 grid((g.nx + 31) / 32, (g.ny + 3) / 4, (g.nz + 1) / 2);  // one thread per pair of planes
    k_collide_stream_far_f32<<<grid, dim3(32, 4), 0, s>>>(g, (const float *)src, (float *)dst, utop_in, utop_out, st,
                                                          slot, hbox, box);
    return cudaGetLastError();
}

}  // namespace turret
