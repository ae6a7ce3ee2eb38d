// support_kernels.cu -- the single-run launch of the support-box moments
// (u*, sigma of Eq. 10 at t + 1) and of the marker binning (block code in
// support_moments.cuh).
#include "support_moments.cuh"

namespace turret {

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
