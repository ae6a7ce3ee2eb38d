// window_kernels.cu -- window operations outside the collide+stream: the
// re-injection copy of Sec. 2.5 (an option beside the ring window, whose
// slide is part of the particle update and of the pull).
#include "turret_internal.cuh"

namespace turret {

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

}  // namespace turret
