// mlp.cu -- the force/torque surrogate network of the particle predictor:
// 34 inputs -> three hidden layers of 128 exact-GELU units -> 6 outputs, on
// standardised inputs and outputs, trained on trajectories the solver logs.
// (Not in the paper, whose only predictor is the orientation
// predictor-corrector of Sec. 2.3; it predicts F(t+1), T(t+1) for the marker
// velocities of the immersed-boundary step, Sec. 2.2.)
//
// Kernels:
//   k_gemm        C = A B with either operand transposed, BF16 tensor-core
//                 mma.sync m16n8k16 with FP32 accumulation (or an FP32
//                 CUDA-core check mode), fused epilogues: bias + GELU
//                 (forward), GELU' product (backward), plain store (weight
//                 gradients).  64x64 tiles, 32-deep K chunks staged in shared
//                 memory; no split-K, no atomics: deterministic.
//   k_mlp_infer   the whole forward pass of up to 16 samples per block, with
//                 activations in shared memory (the predictor's inference).
//   k_loss, k_colsum, k_adamw, k_standardise: loss and its gradient, bias
//                 gradients, AdamW (decoupled weight decay), normalisation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <string>
#include <type_traits>
#include <vector>

#include "../../include/turret.h"
#include "turret_internal.cuh"

using namespace turret;

namespace turret {

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_prime_f(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// ---------------------------------------------------------------------------
// GEMM.  A(m, k) = ta ? A[k * lda + m] : A[m * lda + k];
//        B(k, n) = tb ? B[k * ldb + n] : B[n * ldb + k]   (tb = 0: weights [N][K]).
struct GemmArgs {
    const float *A;
    const float *B;
    float *C;
    const float *bias;  // [N], added when non-null
    float *Aout;        // EPI_GELU: gelu of the result
    const float *Zg;    // EPI_DGELU: the result times gelu'(Zg)
    int lda, ldb, ldc, ldo, ldz;
    int ta, tb;
    int M, N, K;
    int kslice;         // > 0: block z sums K range [z kslice, (z+1) kslice) into part[z][M][N]
    float *part;
};
enum { EPI_STORE = 0, EPI_GELU = 1, EPI_DGELU = 2 };
// split-K of the weight-gradient products (reductions over the batch): slices
// of KSLICE rows, partial sums added in slice order by k_sum_slices
constexpr int KSLICE = 256, MAX_SLICES = 64;
constexpr int GBM = 64, GBN = 64, GBK = 32, GTHREADS = 128;

__device__ __forceinline__ void epilogue(const GemmArgs &g, int epi, int m, int n, float acc) {
    if (m >= g.M || n >= g.N) return;
    if (g.kslice > 0) {  // partial sum of this block's K slice
        g.part[((size_t)blockIdx.z * g.M + m) * g.N + n] = acc;
        return;
    }
    float v = acc + (g.bias ? g.bias[n] : 0.0f);
    if (epi == EPI_DGELU) v *= gelu_prime_f(g.Zg[(size_t)m * g.ldz + n]);
    g.C[(size_t)m * g.ldc + n] = v;
    if (epi == EPI_GELU) g.Aout[(size_t)m * g.ldo + n] = gelu_f(v);
}

template <bool TC>
__global__ void __launch_bounds__(GTHREADS) k_gemm(GemmArgs g, int epi) {
    constexpr int PAD = TC ? 8 : 1;
    using E = typename std::conditional<TC, __nv_bfloat16, float>::type;
    __shared__ __align__(16) E As[GBM][GBK + PAD];
    __shared__ __align__(16) E Bs[GBN][GBK + PAD];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
    const int lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // warp tile origin (TC)
    const int grp = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
    float sacc[4][8];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) sacc[i][j] = 0.0f;
    const int kbeg = g.kslice > 0 ? blockIdx.z * g.kslice : 0;
    const int kend = g.kslice > 0 ? min(g.K, kbeg + g.kslice) : g.K;
    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
        // stage the A and B tiles (any layout -> [row][k]), zero outside the matrices
#pragma unroll 4
        for (int e = tid; e < GBM * GBK; e += GTHREADS) {
            int m, k;
            if (g.ta) { k = e / GBM; m = e % GBM; } else { m = e / GBK; k = e % GBK; }
            const int gm = m0 + m, gk = k0 + k;
            float v = 0.0f;
            if (gm < g.M && gk < kend) v = g.ta ? g.A[(size_t)gk * g.lda + gm] : g.A[(size_t)gm * g.lda + gk];
            if constexpr (TC) As[m][k] = __float2bfloat16_rn(v); else As[m][k] = v;
        }
#pragma unroll 4
        for (int e = tid; e < GBN * GBK; e += GTHREADS) {
            int n, k;
            if (g.tb) { k = e / GBN; n = e % GBN; } else { n = e / GBK; k = e % GBK; }
            const int gn = n0 + n, gk = k0 + k;
            float v = 0.0f;
            if (gn < g.N && gk < kend) v = g.tb ? g.B[(size_t)gk * g.ldb + gn] : g.B[(size_t)gn * g.ldb + gk];
            if constexpr (TC) Bs[n][k] = __float2bfloat16_rn(v); else Bs[n][k] = v;
        }
        __syncthreads();
        if constexpr (TC) {
#pragma unroll
            for (int kk = 0; kk < GBK; kk += 16) {
                uint32_t a[2][4], b[4][2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int r = wm + 16 * i + grp;
                    a[i][0] = ld_pair(&As[r][kk + 2 * tig]);
                    a[i][1] = ld_pair(&As[r + 8][kk + 2 * tig]);
                    a[i][2] = ld_pair(&As[r][kk + 8 + 2 * tig]);
                    a[i][3] = ld_pair(&As[r + 8][kk + 8 + 2 * tig]);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = wn + 8 * j + grp;
                    b[j][0] = ld_pair(&Bs[c][kk + 2 * tig]);
                    b[j][1] = ld_pair(&Bs[c][kk + 8 + 2 * tig]);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
            }
        } else {
            const int tr = tid >> 3, tc = tid & 7;  // rows 4 tr + i, columns tc + 8 j
#pragma unroll 4
            for (int k = 0; k < GBK; ++k)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) sacc[i][j] = fmaf(As[4 * tr + i][k], Bs[tc + 8 * j][k], sacc[i][j]);
        }
        __syncthreads();
    }
    if constexpr (TC) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = m0 + wm + 16 * i + grp, c = n0 + wn + 8 * j + 2 * tig;
                epilogue(g, epi, r, c, acc[i][j][0]);
                epilogue(g, epi, r, c + 1, acc[i][j][1]);
                epilogue(g, epi, r + 8, c, acc[i][j][2]);
                epilogue(g, epi, r + 8, c + 1, acc[i][j][3]);
            }
    } else {
        const int tr = tid >> 3, tc = tid & 7;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) epilogue(g, epi, m0 + 4 * tr + i, n0 + tc + 8 * j, sacc[i][j]);
    }
}

// ---------------------------------------------------------------------------
// Standardisation: x_s = (x - mean) / std (inputs and targets), and back.
__global__ void k_standardise(const float *__restrict__ x, int n, int d, const float *__restrict__ mean,
                              const float *__restrict__ stdv, float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * d) return;
    const int c = i % d;
    out[i] = (x[i] - mean[c]) / stdv[c];
}

__global__ void k_unstandardise(const float *__restrict__ y, int n, const float *__restrict__ mean,
                                const float *__restrict__ stdv, float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * MLP_OUT) return;
    const int c = i % MLP_OUT;
    out[i] = fmaf(y[i], stdv[c], mean[c]);
}

// Loss = mean over samples and outputs of (y - t)^2 (accumulated in FP64 in a
// fixed order) and dL/dy = 2 (y - t) / (6 n).
constexpr int LOSS_THREADS = 256;
__global__ void __launch_bounds__(LOSS_THREADS) k_loss(const float *__restrict__ y, const float *__restrict__ t,
                                                       int n, float *__restrict__ dy, double *__restrict__ loss) {
    __shared__ double part[LOSS_THREADS];
    const int total = n * MLP_OUT;
    const float sc = 2.0f / (float)total;
    double s = 0.0;
    for (int i = threadIdx.x; i < total; i += LOSS_THREADS) {
        const float e = y[i] - t[i];
        s += (double)e * (double)e;
        dy[i] = sc * e;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = LOSS_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] / (double)total;
}

// Bias gradient, first pass: column sums of dZ [n][ld] over the rows of
// slice blockIdx.y (KSLICE rows, in row order) into part[slice][ncol].
__global__ void k_colsum(const float *__restrict__ dz, int n, int ncol, int ld, float *__restrict__ part) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    const int r0 = blockIdx.y * KSLICE, r1 = min(n, r0 + KSLICE);
    float s = 0.0f;
    for (int r = r0; r < r1; ++r) s += dz[(size_t)r * ld + c];
    part[(size_t)blockIdx.y * ncol + c] = s;
}

// Sum of nsl partial results part[z][count] in slice order z = 0, 1, ...
__global__ void k_sum_slices(const float *__restrict__ part, int nsl, int count, float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = part[i];
    for (int z = 1; z < nsl; ++z) s += part[(size_t)z * count + i];
    out[i] = s;
}

// Offsets of the flat parameter vector (W1 b1 W2 b2 W3 b3 W4 b4).
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H, OFF_B2 = OFF_W2 + MLP_H * MLP_H,
              OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_H * MLP_H, OFF_W4 = OFF_B3 + MLP_H,
              OFF_B4 = OFF_W4 + MLP_OUT * MLP_H, OFF_END = OFF_B4 + MLP_OUT;
static_assert(OFF_END == MLP_NPARAM, "parameter layout");

__device__ __forceinline__ bool is_weight(int i) {
    return i < OFF_B1 || (i >= OFF_W2 && i < OFF_B2) || (i >= OFF_W3 && i < OFF_B3) || (i >= OFF_W4 && i < OFF_B4);
}

// BF16 copies of the weight matrices in the padded layout of the inference
// kernel: W1 [128][48] (columns 34..47 zero), W2, W3 [128][128], W4 [8][128]
// (rows 6, 7 zero).
constexpr int WB1 = 0, WB2 = WB1 + MLP_H * MLP_INP, WB3 = WB2 + MLP_H * MLP_H, WB4 = WB3 + MLP_H * MLP_H,
              WB_END = WB4 + MLP_OUTP * MLP_H;

__global__ void k_refresh_bf16(const float *__restrict__ P, __nv_bfloat16 *__restrict__ wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= WB_END) return;
    float v = 0.0f;
    if (i < WB2) {
        const int r = i / MLP_INP, c = i % MLP_INP;
        v = c < MLP_IN ? P[OFF_W1 + r * MLP_IN + c] : 0.0f;
    } else if (i < WB3) {
        v = P[OFF_W2 + (i - WB2)];
    } else if (i < WB4) {
        v = P[OFF_W3 + (i - WB3)];
    } else {
        const int r = (i - WB4) / MLP_H, c = (i - WB4) % MLP_H;
        v = r < MLP_OUT ? P[OFF_W4 + r * MLP_H + c] : 0.0f;
    }
    wb[i] = __float2bfloat16_rn(v);
}

// AdamW (Loshchilov & Hutter): moments, bias correction, decoupled decay of
// the weight matrices.
__global__ void k_adamw(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ Mm,
                        float *__restrict__ Vv, float lr, float b1, float b2, float eps, float wd, float bc1,
                        float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NPARAM) return;
    const float g = G[i];
    const float m = b1 * Mm[i] + (1.0f - b1) * g;
    const float v = b2 * Vv[i] + (1.0f - b2) * g * g;
    Mm[i] = m;
    Vv[i] = v;
    const float p = P[i];
    const float upd = (m / bc1) / (sqrtf(v / bc2) + eps) + (is_weight(i) ? wd * p : 0.0f);
    P[i] = p - lr * upd;
}

// ---------------------------------------------------------------------------
// Inference of up to 16 samples per block (the predictor): features
// standardised, four layers with activations in shared memory, outputs
// de-standardised.  TC: BF16 tensor cores with the padded BF16 weights (the
// same operands and k order as k_gemm, hence the same results); otherwise
// FP32 on the CUDA cores with the FP32 weights.
constexpr int INF_ROWS = 16, INF_THREADS = 128, ACT_LD = MLP_H + 8;

template <bool TC>
__device__ __forceinline__ void infer_layer(const MlpDev &w, int layer, const float (*actf)[ACT_LD],
                                            const __nv_bfloat16 (*actb)[ACT_LD], float (*outf)[ACT_LD],
                                            __nv_bfloat16 (*outb)[ACT_LD], int nrows) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = layer == 0 ? MLP_IN : MLP_H;
    const int N = layer == 3 ? MLP_OUT : MLP_H;
    const float *bias = w.P + (layer == 0 ? OFF_B1 : layer == 1 ? OFF_B2 : layer == 2 ? OFF_B3 : OFF_B4);
    if constexpr (TC) {
        const __nv_bfloat16 *W = w.Wb + (layer == 0 ? WB1 : layer == 1 ? WB2 : layer == 2 ? WB3 : WB4);
        const int ldw = layer == 0 ? MLP_INP : MLP_H;
        const int Kp = layer == 0 ? MLP_INP : MLP_H;
        const int ntile = layer == 3 ? 1 : 4;  // n8 tiles per warp
        if (layer == 3 && warp > 0) return;
        const int grp = lane >> 2, tig = lane & 3;
        float acc[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[j][q] = 0.0f;
        for (int kk = 0; kk < Kp; kk += 16) {
            uint32_t a[4];
            a[0] = ld_pair(&actb[grp][kk + 2 * tig]);
            a[1] = ld_pair(&actb[grp + 8][kk + 2 * tig]);
            a[2] = ld_pair(&actb[grp][kk + 8 + 2 * tig]);
            a[3] = ld_pair(&actb[grp + 8][kk + 8 + 2 * tig]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j >= ntile) break;
                const int c = 32 * warp + 8 * j + grp;
                uint32_t b[2];
                b[0] = ld_pair(W + (size_t)c * ldw + kk + 2 * tig);
                b[1] = ld_pair(W + (size_t)c * ldw + kk + 8 + 2 * tig);
                mma_bf16(acc[j], a, b);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j >= ntile) break;
            const int c = 32 * warp + 8 * j + 2 * tig;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = grp + (q >= 2 ? 8 : 0), cc = c + (q & 1);
                if (cc < N) {
                    const float z = acc[j][q] + bias[cc];
                    const float v = layer == 3 ? z : gelu_f(z);
                    outf[r][cc] = v;
                    outb[r][cc] = __float2bfloat16_rn(v);
                }
            }
        }
    } else {
        const float *W = w.P + (layer == 0 ? OFF_W1 : layer == 1 ? OFF_W2 : layer == 2 ? OFF_W3 : OFF_W4);
        for (int e = tid; e < INF_ROWS * N; e += INF_THREADS) {
            const int r = e / N, c = e % N;
            float s = 0.0f;
            for (int k = 0; k < K; ++k) s = fmaf(actf[r][k], W[(size_t)c * K + k], s);
            const float z = s + bias[c];
            const float v = layer == 3 ? z : gelu_f(z);
            outf[r][c] = v;
            outb[r][c] = __float2bfloat16_rn(v);
        }
    }
    (void)nrows;
}

struct InferSmem {
    float af[2][INF_ROWS][ACT_LD];
    __align__(16) __nv_bfloat16 ab[2][INF_ROWS][ACT_LD];
};

template <bool TC>
__device__ __forceinline__ void mlp_infer_rows(const MlpDev &w, const float *__restrict__ x, int n, int row0,
                                               float *__restrict__ y, InferSmem &sm) {
    float (*af)[INF_ROWS][ACT_LD] = sm.af;
    __nv_bfloat16 (*ab)[INF_ROWS][ACT_LD] = sm.ab;
    const int tid = threadIdx.x;
    const int nrows = min(INF_ROWS, n - row0);
    for (int e = tid; e < INF_ROWS * ACT_LD; e += INF_THREADS) {
        const int r = e / ACT_LD, c = e % ACT_LD;
        float v = 0.0f;
        if (r < nrows && c < MLP_IN) v = (x[(size_t)(row0 + r) * MLP_IN + c] - w.mean_x[c]) / w.std_x[c];
        af[0][r][c] = v;
        ab[0][r][c] = __float2bfloat16_rn(v);
        af[1][r][c] = 0.0f;
        ab[1][r][c] = __float2bfloat16_rn(0.0f);
    }
    __syncthreads();
    for (int l = 0; l < 4; ++l) {
        const int s = l & 1;
        infer_layer<TC>(w, l, af[s], ab[s], af[s ^ 1], ab[s ^ 1], nrows);
        __syncthreads();
    }
    for (int e = tid; e < nrows * MLP_OUT; e += INF_THREADS) {
        const int r = e / MLP_OUT, c = e % MLP_OUT;
        y[(size_t)(row0 + r) * MLP_OUT + c] = fmaf(af[0][r][c], w.std_y[c], w.mean_y[c]);
    }
}

template <bool TC>
__global__ void __launch_bounds__(INF_THREADS) k_mlp_infer(MlpDev w, const float *__restrict__ x, int n,
                                                           float *__restrict__ y) {
    __shared__ InferSmem sm;
    mlp_infer_rows<TC>(w, x, n, blockIdx.x * INF_ROWS, y, sm);
}

// ---------------------------------------------------------------------------
// Features of the predictor at time level t (all in the body frame of t,
// whose axes are the rows d_0, d_1, d_2 of the orientation matrix M):
//   [0:4]   unit quaternion (w, x, y, z), w >= 0, of M, by Shepperd's method
//           (S. W. Shepperd, J. Guidance and Control 1 (1978) 223): the
//           largest of 1 + tr M, 1 + 2 M_ii - tr M picks the stable formula
//   [4:7]   M v(t - 1/2)          [7:10]  M w(t - 1/2)
//   [10:34] M F(t - h) / sF, M T(t - h) / sT for h = 0, 1, 2, 3, with the
//           scales sF = max_h |F(t - h)|, sT = max_h |T(t - h)| (1 if zero)
// Targets: the departure of the next force and torque from their linear
// extrapolation, in the same frame and scale:
//   M (F(t+1) - 2 F(t) + F(t-1)) / sF,  M (T(t+1) - 2 T(t) + T(t-1)) / sT,
// so the prediction is F^ = 2 F(t) - F(t-1) + sF M^T y (and T^ alike): the
// network corrects linear extrapolation, independent of the force's size.
__device__ void quat_of(const double *M, double q[4]) {
    const double tr = M[0] + M[4] + M[8];
    const double c[4] = {1.0 + tr, 1.0 + 2.0 * M[0] - tr, 1.0 + 2.0 * M[4] - tr, 1.0 + 2.0 * M[8] - tr};
    int b = 0;
    for (int i = 1; i < 4; ++i)
        if (c[i] > c[b]) b = i;
    const double s = 2.0 * sqrt(c[b]);  // = 4 |q_b|
    const double r = 1.0 / s;
    if (b == 0) {
        q[0] = 0.25 * s; q[1] = (M[7] - M[5]) * r; q[2] = (M[2] - M[6]) * r; q[3] = (M[3] - M[1]) * r;
    } else if (b == 1) {
        q[0] = (M[7] - M[5]) * r; q[1] = 0.25 * s; q[2] = (M[1] + M[3]) * r; q[3] = (M[2] + M[6]) * r;
    } else if (b == 2) {
        q[0] = (M[2] - M[6]) * r; q[1] = (M[1] + M[3]) * r; q[2] = 0.25 * s; q[3] = (M[5] + M[7]) * r;
    } else {
        q[0] = (M[3] - M[1]) * r; q[1] = (M[2] + M[6]) * r; q[2] = (M[5] + M[7]) * r; q[3] = 0.25 * s;
    }
    if (q[0] < 0.0)
        for (int i = 0; i < 4; ++i) q[i] = -q[i];
}

__device__ __forceinline__ void to_body(const double *M, const double *a, double scale, float *out) {
    for (int i = 0; i < 3; ++i) out[i] = (float)((M[3 * i] * a[0] + M[3 * i + 1] * a[1] + M[3 * i + 2] * a[2]) / scale);
}

__device__ void scales_of(const double (*Fh)[3], const double (*Th)[3], double &sF, double &sT) {
    sF = 0.0;
    sT = 0.0;
    for (int h = 0; h < 4; ++h) {
        sF = fmax(sF, sqrt(Fh[h][0] * Fh[h][0] + Fh[h][1] * Fh[h][1] + Fh[h][2] * Fh[h][2]));
        sT = fmax(sT, sqrt(Th[h][0] * Th[h][0] + Th[h][1] * Th[h][1] + Th[h][2] * Th[h][2]));
    }
    if (!(sF > 0.0)) sF = 1.0;
    if (!(sT > 0.0)) sT = 1.0;
}

__device__ void features_of(const double *M, const double *v, const double *w, const double (*Fh)[3],
                            const double (*Th)[3], float *x) {
    double q[4], sF, sT;
    quat_of(M, q);
    scales_of(Fh, Th, sF, sT);
    for (int i = 0; i < 4; ++i) x[i] = (float)q[i];
    to_body(M, v, 1.0, x + 4);
    to_body(M, w, 1.0, x + 7);
    for (int h = 0; h < 4; ++h) {
        to_body(M, Fh[h], sF, x + 10 + 6 * h);
        to_body(M, Th[h], sT, x + 13 + 6 * h);
    }
}

// Prediction of F(t+1), T(t+1) at the start of the step t -> t+1 (slot =
// the window slot of t).  Linear extrapolation 2 F(t) - F(t-1) in mode 1, and
// in mode 2 while fewer than four history levels exist or while the
// network's own previous prediction missed by more than the threshold (the
// fallback); the network, in mode 2, runs whenever four levels exist, so its
// accuracy keeps being checked while it is not used.
__device__ void predict_block(const MlpDev &w, bool has_net, DevState *st, int slot, int mode, InferSmem &sm) {
    __shared__ int run_net;
    Predictor &P = st->pr;
    if (threadIdx.x == 0) {
        for (int q = 0; q < 3; ++q) {
            P.Fhat[q] = P.hist_n >= 2 ? 2.0 * P.Fh[0][q] - P.Fh[1][q] : P.Fh[0][q];
            P.That[q] = P.hist_n >= 2 ? 2.0 * P.Th[0][q] - P.Th[1][q] : P.Th[0][q];
        }
        P.predicted = 1;
        P.by_net = 0;
        P.steps += 1;
        run_net = mode == 2 && has_net && P.hist_n >= 4;
        if (run_net) {
            const BodySlot &S = st->s[slot];
            features_of(S.d, S.v, S.w, P.Fh, P.Th, P.feat);
        } else if (mode == 2) {
            P.fallbacks += 1;
        }
    }
    __syncthreads();
    if (!run_net) return;
    if (w.precision == 0) mlp_infer_rows<true>(w, P.feat, 1, 0, P.yb, sm);
    else mlp_infer_rows<false>(w, P.feat, 1, 0, P.yb, sm);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double *M = st->s[slot].d;
        double sF, sT;
        scales_of(P.Fh, P.Th, sF, sT);
        for (int i = 0; i < 3; ++i) {  // linear extrapolation + scale * M^T y
            P.Fnet[i] = 2.0 * P.Fh[0][i] - P.Fh[1][i] + sF * (M[i] * P.yb[0] + M[3 + i] * P.yb[1] + M[6 + i] * P.yb[2]);
            P.Tnet[i] = 2.0 * P.Th[0][i] - P.Th[1][i] + sT * (M[i] * P.yb[3] + M[3 + i] * P.yb[4] + M[6 + i] * P.yb[5]);
        }
        P.net_ok = 1;
        if (!P.fallback) {
            for (int i = 0; i < 3; ++i) {
                P.Fhat[i] = P.Fnet[i];
                P.That[i] = P.Tnet[i];
            }
            P.by_net = 1;
            P.mlp_steps += 1;
        } else {
            P.fallbacks += 1;
        }
    }
}

__global__ void __launch_bounds__(INF_THREADS) k_predict(MlpDev w, int has_net, DevState *st, int slot, int mode) {
    __shared__ InferSmem sm;
    predict_block(w, has_net != 0, st, slot, mode, sm);
}

__global__ void __launch_bounds__(INF_THREADS) k_batch_predict(const RunDesc *__restrict__ runs, int slot) {
    __shared__ InferSmem sm;
    const RunDesc &R = runs[blockIdx.x];
    if (R.bc.predictor == 0) return;
    predict_block(R.mlp, R.mlp.P != nullptr, R.st, slot, R.bc.predictor, sm);
}

cudaError_t launch_predict(const MlpDev *w, DevState *st, int slot, int mode, cudaStream_t s) {
    MlpDev v;
    memset(&v, 0, sizeof v);
    if (w) v = *w;
    k_predict<<<1, INF_THREADS, 0, s>>>(v, w != nullptr, st, slot, mode);
    return cudaGetLastError();
}

cudaError_t launch_batch_predict(const RunDesc *runs, int nruns, int slot, cudaStream_t s) {
    k_batch_predict<<<nruns, INF_THREADS, 0, s>>>(runs, slot);
    return cudaGetLastError();
}

// Training pairs from a trajectory log of consecutive time levels (records
// as written by the force reduction): sample j uses records j .. j + 4
// (history t - 3 .. t with t = j + 3, target t + 1).  Records whose time
// levels are not consecutive give NaN features (and count in *bad).
__global__ void k_build_samples(const double *__restrict__ log, long long nsamp, float *__restrict__ x,
                                float *__restrict__ y, int *bad) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nsamp) return;
    const double *r[5];
    for (int h = 0; h < 5; ++h) r[h] = log + (size_t)(j + h) * LOG_REC;  // r[3] = t, r[4] = t + 1
    bool ok = true;
    for (int h = 1; h < 5; ++h) ok = ok && r[h][21] == r[h - 1][21] + 1.0;
    double Fh[4][3], Th[4][3];
    for (int h = 0; h < 4; ++h)
        for (int q = 0; q < 3; ++q) {
            Fh[h][q] = r[3 - h][15 + q];
            Th[h][q] = r[3 - h][18 + q];
        }
    float *xo = x + (size_t)j * MLP_IN;
    features_of(r[3], r[3] + 9, r[3] + 12, Fh, Th, xo);
    double sF, sT, dF[3], dT[3];
    scales_of(Fh, Th, sF, sT);
    for (int q = 0; q < 3; ++q) {  // departure of t + 1 from the linear extrapolation
        dF[q] = r[4][15 + q] - 2.0 * Fh[0][q] + Fh[1][q];
        dT[q] = r[4][18 + q] - 2.0 * Th[0][q] + Th[1][q];
    }
    to_body(r[3], dF, sF, y + (size_t)j * MLP_OUT);
    to_body(r[3], dT, sT, y + (size_t)j * MLP_OUT + 3);
    if (!ok) {
        for (int i = 0; i < MLP_IN; ++i) xo[i] = NAN;
        atomicAdd(bad, 1);
    }
}

cudaError_t launch_mlp_infer(const MlpDev &w, const float *x, int n, float *y, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nb = (n + INF_ROWS - 1) / INF_ROWS;
    if (w.precision == 0) k_mlp_infer<true><<<nb, INF_THREADS, 0, s>>>(w, x, n, y);
    else k_mlp_infer<false><<<nb, INF_THREADS, 0, s>>>(w, x, n, y);
    return cudaGetLastError();
}

}  // namespace turret

// ===========================================================================
// Host object behind turret_mlp.
struct turret_mlp {
    int cap, precision;
    cudaStream_t stream;
    MlpDev dev;
    float *P, *G, *Mm, *Vv;
    __nv_bfloat16 *Wb;
    float *norm;  // mean_x [34], std_x [34], mean_y [6], std_y [6]
    float *X0, *T, *Y, *dY, *Z[3], *A[3], *D[2];
    float *part;  // split-K partial sums [MAX_SLICES][128][128]
    double *loss;
    long long adam_step;
    // the training step (standardise, forward, backward, AdamW, BF16 copy) as
    // one CUDA graph per batch size; between replays only the input pointers
    // and the optimiser's scalars change, in the three nodes that take them
    cudaGraph_t train_graph;  // kept: its nodes address the instantiated graph's nodes
    cudaGraphExec_t train_exec;
    int train_n;
    cudaGraphNode_t node_x, node_y, node_adam;
    std::string err;
};

namespace {
std::string g_mlp_err;

struct MCarver {
    char *base;
    size_t off;
    void *take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

void carve_mlp(MCarver &cv, int cap, turret_mlp *m) {
    turret_mlp t;
    turret_mlp &M = m ? *m : t;
    M.P = (float *)cv.take(MLP_NPARAM * 4);
    M.G = (float *)cv.take(MLP_NPARAM * 4);
    M.Mm = (float *)cv.take(MLP_NPARAM * 4);
    M.Vv = (float *)cv.take(MLP_NPARAM * 4);
    M.Wb = (__nv_bfloat16 *)cv.take(WB_END * 2);
    M.norm = (float *)cv.take(2 * (MLP_IN + MLP_OUT) * 4);
    const size_t c = (size_t)cap;
    M.X0 = (float *)cv.take(c * MLP_IN * 4);
    M.T = (float *)cv.take(c * MLP_OUT * 4);
    M.Y = (float *)cv.take(c * MLP_OUT * 4);
    M.dY = (float *)cv.take(c * MLP_OUT * 4);
    for (int l = 0; l < 3; ++l) {
        M.Z[l] = (float *)cv.take(c * MLP_H * 4);
        M.A[l] = (float *)cv.take(c * MLP_H * 4);
    }
    for (int l = 0; l < 2; ++l) M.D[l] = (float *)cv.take(c * MLP_H * 4);
    M.loss = (double *)cv.take(8);
    M.part = (float *)cv.take((size_t)MAX_SLICES * MLP_H * MLP_H * 4);
}

turret_status mfail(turret_mlp *m, turret_status s, const std::string &msg) {
    if (m) m->err = msg; else g_mlp_err = msg;
    if (s == TURRET_ECUDA) cudaGetLastError();  // a non-sticky error must not surface in later launches
    return s;
}

#define MK(call, where)                                                                                       \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess) return mfail(m, TURRET_ECUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

cudaError_t gemm(const turret_mlp *m, const GemmArgs &g, int epi) {
    const dim3 grid((g.M + GBM - 1) / GBM, (g.N + GBN - 1) / GBN,
                    g.kslice > 0 ? (g.K + g.kslice - 1) / g.kslice : 1);
    if (m->precision == 0) k_gemm<true><<<grid, GTHREADS, 0, m->stream>>>(g, epi);
    else k_gemm<false><<<grid, GTHREADS, 0, m->stream>>>(g, epi);
    return cudaGetLastError();
}

GemmArgs gargs(const float *A, int lda, int ta, const float *B, int ldb, int tb, float *C, int ldc, int M, int N,
               int K) {
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.A = A; g.lda = lda; g.ta = ta;
    g.B = B; g.ldb = ldb; g.tb = tb;
    g.C = C; g.ldc = ldc;
    g.M = M; g.N = N; g.K = K;
    return g;
}

// Forward pass of n standardised rows in X0 -> Y (keeps Z, A for backprop).
cudaError_t forward(turret_mlp *m, int n) {
    const float *W[4] = {m->P + OFF_W1, m->P + OFF_W2, m->P + OFF_W3, m->P + OFF_W4};
    const float *b[4] = {m->P + OFF_B1, m->P + OFF_B2, m->P + OFF_B3, m->P + OFF_B4};
    const float *in = m->X0;
    int K = MLP_IN;
    for (int l = 0; l < 3; ++l) {
        GemmArgs g = gargs(in, K, 0, W[l], K, 0, m->Z[l], MLP_H, n, MLP_H, K);
        g.bias = b[l];
        g.Aout = m->A[l];
        g.ldo = MLP_H;
        cudaError_t e = gemm(m, g, EPI_GELU);
        if (e != cudaSuccess) return e;
        in = m->A[l];
        K = MLP_H;
    }
    GemmArgs g = gargs(in, MLP_H, 0, W[3], MLP_H, 0, m->Y, MLP_OUT, n, MLP_OUT, MLP_H);
    g.bias = b[3];
    return gemm(m, g, EPI_STORE);
}

// Loss of the standardised targets in T and the gradient into G.
cudaError_t backward(turret_mlp *m, int n) {
    cudaError_t e;
    k_loss<<<1, LOSS_THREADS, 0, m->stream>>>(m->Y, m->T, n, m->dY, m->loss);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int offW[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4}, offB[4] = {OFF_B1, OFF_B2, OFF_B3, OFF_B4};
    const int kin[4] = {MLP_IN, MLP_H, MLP_H, MLP_H};
    const float *acts[4] = {m->X0, m->A[0], m->A[1], m->A[2]};
    const float *dz = m->dY;  // gradient of the current layer's output
    int nout = MLP_OUT;
    for (int l = 3; l >= 0; --l) {
        // dW_l = dz^T a_{l-1} ([nout][kin]), db_l = column sums of dz; both
        // reduce over the batch: KSLICE-row slices, partial sums added in order
        const int nsl = (n + KSLICE - 1) / KSLICE;
        GemmArgs g = gargs(dz, nout, 1, acts[l], kin[l], 1, m->G + offW[l], kin[l], nout, kin[l], n);
        g.kslice = KSLICE;
        g.part = m->part;
        if ((e = gemm(m, g, EPI_STORE)) != cudaSuccess) return e;
        k_sum_slices<<<(nout * kin[l] + 255) / 256, 256, 0, m->stream>>>(m->part, nsl, nout * kin[l], m->G + offW[l]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_colsum<<<dim3((nout + 127) / 128, nsl), 128, 0, m->stream>>>(dz, n, nout, nout, m->part);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_sum_slices<<<(nout + 255) / 256, 256, 0, m->stream>>>(m->part, nsl, nout, m->G + offB[l]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (l == 0) break;
        // dz_{l-1} = (dz W_l) * gelu'(z_{l-1})
        float *dst = m->D[l & 1];
        GemmArgs h = gargs(dz, nout, 0, m->P + offW[l], kin[l], 1, dst, MLP_H, n, MLP_H, nout);
        h.Zg = m->Z[l - 1];
        h.ldz = MLP_H;
        if ((e = gemm(m, h, EPI_DGELU)) != cudaSuccess) return e;
        dz = dst;
        nout = MLP_H;
    }
    return cudaSuccess;
}

cudaError_t prepare(turret_mlp *m, const float *x, const float *y, int n) {
    k_standardise<<<(n * MLP_IN + 255) / 256, 256, 0, m->stream>>>(x, n, MLP_IN, m->norm, m->norm + MLP_IN, m->X0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !y) return e;
    k_standardise<<<(n * MLP_OUT + 255) / 256, 256, 0, m->stream>>>(y, n, MLP_OUT, m->norm + 2 * MLP_IN,
                                                                    m->norm + 2 * MLP_IN + MLP_OUT, m->T);
    return cudaGetLastError();
}

cudaError_t refresh(turret_mlp *m) {
    k_refresh_bf16<<<(WB_END + 255) / 256, 256, 0, m->stream>>>(m->P, m->Wb);
    return cudaGetLastError();
}

}  // namespace

extern "C" size_t mlp_workspace_bytes(int32_t batch_cap) {
    if (batch_cap < 1 || batch_cap > MAX_SLICES * KSLICE) return 0;
    MCarver cv{nullptr, 0};
    carve_mlp(cv, batch_cap, nullptr);
    return cv.off + 256;
}

extern "C" turret_status mlp_init(turret_mlp **out, int32_t batch_cap, int32_t precision, const float *params,
                                  void *ws, size_t ws_bytes, void *stream) {
    turret_mlp *m = nullptr;
    if (!out) return mfail(m, TURRET_EINVAL, "out is NULL");
    *out = nullptr;
    if (precision < 0 || precision > 1) return mfail(m, TURRET_EINVAL, "precision must be 0 (bf16) or 1 (fp32)");
    const size_t need = mlp_workspace_bytes(batch_cap);
    if (need == 0) return mfail(m, TURRET_EINVAL, "invalid batch capacity");
    if (!params) return mfail(m, TURRET_EINVAL, "NULL parameters");
    if (!ws || ws_bytes < need) return mfail(m, TURRET_ENOMEM, "mlp workspace too small");
    if (((uintptr_t)ws & 255) != 0) return mfail(m, TURRET_EINVAL, "workspace must be 256-byte aligned");
    m = new turret_mlp();
    m->cap = batch_cap;
    m->precision = precision;
    m->stream = (cudaStream_t)stream;
    m->adam_step = 0;
    m->train_exec = nullptr;
    m->train_graph = nullptr;
    m->train_n = 0;
    MCarver cv{(char *)ws, 0};
    carve_mlp(cv, batch_cap, m);
    std::vector<float> norm(2 * (MLP_IN + MLP_OUT));
    for (int i = 0; i < MLP_IN; ++i) norm[MLP_IN + i] = 1.0f;                 // std_x
    for (int i = 0; i < MLP_OUT; ++i) norm[2 * MLP_IN + MLP_OUT + i] = 1.0f;  // std_y
    cudaError_t e = cudaMemcpyAsync(m->P, params, MLP_NPARAM * 4, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->Mm, 0, MLP_NPARAM * 4, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->Vv, 0, MLP_NPARAM * 4, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->norm, norm.data(), norm.size() * 4, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = refresh(m);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        delete m;
        return mfail(nullptr, TURRET_ECUDA, std::string("mlp_init: ") + cudaGetErrorString(e));
    }
    m->dev.P = m->P;
    m->dev.Wb = m->Wb;
    m->dev.mean_x = m->norm;
    m->dev.std_x = m->norm + MLP_IN;
    m->dev.mean_y = m->norm + 2 * MLP_IN;
    m->dev.std_y = m->norm + 2 * MLP_IN + MLP_OUT;
    m->dev.precision = precision;
    *out = m;
    return TURRET_OK;
}

extern "C" turret_status mlp_set_params(turret_mlp *m, const float *params) {
    if (!m || !params) return mfail(m, TURRET_EINVAL, "NULL argument");
    MK(cudaMemcpyAsync(m->P, params, MLP_NPARAM * 4, cudaMemcpyHostToDevice, m->stream), "set params");
    MK(refresh(m), "refresh bf16");
    MK(cudaStreamSynchronize(m->stream), "set params sync");
    return TURRET_OK;
}

extern "C" turret_status mlp_get_params(turret_mlp *m, float *params) {
    if (!m || !params) return mfail(m, TURRET_EINVAL, "NULL argument");
    MK(cudaMemcpyAsync(params, m->P, MLP_NPARAM * 4, cudaMemcpyDeviceToHost, m->stream), "get params");
    MK(cudaStreamSynchronize(m->stream), "get params sync");
    return TURRET_OK;
}

extern "C" turret_status mlp_set_norm(turret_mlp *m, const float *mean_x, const float *std_x, const float *mean_y,
                                      const float *std_y) {
    if (!m || !mean_x || !std_x || !mean_y || !std_y) return mfail(m, TURRET_EINVAL, "NULL argument");
    std::vector<float> h(2 * (MLP_IN + MLP_OUT));
    for (int i = 0; i < MLP_IN; ++i) {
        if (!(std_x[i] > 0.0f)) return mfail(m, TURRET_EINVAL, "non-positive std");
        h[i] = mean_x[i];
        h[MLP_IN + i] = std_x[i];
    }
    for (int i = 0; i < MLP_OUT; ++i) {
        if (!(std_y[i] > 0.0f)) return mfail(m, TURRET_EINVAL, "non-positive std");
        h[2 * MLP_IN + i] = mean_y[i];
        h[2 * MLP_IN + MLP_OUT + i] = std_y[i];
    }
    MK(cudaMemcpyAsync(m->norm, h.data(), h.size() * 4, cudaMemcpyHostToDevice, m->stream), "set norm");
    MK(cudaStreamSynchronize(m->stream), "set norm sync");
    return TURRET_OK;
}

extern "C" turret_status mlp_forward(turret_mlp *m, const float *x, int32_t n, float *y) {
    if (!m || !x || !y) return mfail(m, TURRET_EINVAL, "NULL argument");
    if (n < 1 || n > m->cap) return mfail(m, TURRET_EINVAL, "batch outside 1..capacity");
    MK(prepare(m, x, nullptr, n), "standardise");
    MK(forward(m, n), "forward");
    k_unstandardise<<<(n * MLP_OUT + 255) / 256, 256, 0, m->stream>>>(m->Y, n, m->dev.mean_y, m->dev.std_y, y);
    MK(cudaGetLastError(), "unstandardise");
    return TURRET_OK;
}

extern "C" turret_status mlp_infer(turret_mlp *m, const float *x, int32_t n, float *y) {
    if (!m || !x || !y) return mfail(m, TURRET_EINVAL, "NULL argument");
    if (n < 1) return mfail(m, TURRET_EINVAL, "empty batch");
    MK(launch_mlp_infer(m->dev, x, n, y, m->stream), "infer");
    return TURRET_OK;
}

extern "C" turret_status mlp_loss_grad(turret_mlp *m, const float *x, const float *y, int32_t n, float *loss,
                                       float *grad) {
    if (!m || !x || !y || !loss) return mfail(m, TURRET_EINVAL, "NULL argument");
    if (n < 1 || n > m->cap) return mfail(m, TURRET_EINVAL, "batch outside 1..capacity");
    MK(prepare(m, x, y, n), "standardise");
    MK(forward(m, n), "forward");
    MK(backward(m, n), "backward");
    double L = 0.0;
    MK(cudaMemcpyAsync(&L, m->loss, 8, cudaMemcpyDeviceToHost, m->stream), "loss");
    if (grad) MK(cudaMemcpyAsync(grad, m->G, MLP_NPARAM * 4, cudaMemcpyDeviceToDevice, m->stream), "grad");
    MK(cudaStreamSynchronize(m->stream), "loss sync");
    *loss = (float)L;
    return TURRET_OK;
}

namespace {
// One training step's kernels on the network's stream.
cudaError_t enqueue_train(turret_mlp *m, const float *x, const float *y, int n, const turret_adamw *opt, float bc1,
                          float bc2) {
    cudaError_t e = prepare(m, x, y, n);
    if (e == cudaSuccess) e = forward(m, n);
    if (e == cudaSuccess) e = backward(m, n);
    if (e != cudaSuccess) return e;
    k_adamw<<<(MLP_NPARAM + 255) / 256, 256, 0, m->stream>>>(m->P, m->G, m->Mm, m->Vv, opt->lr, opt->beta1,
                                                             opt->beta2, opt->eps, opt->weight_decay, bc1, bc2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return refresh(m);
}

void drop_train_graph(turret_mlp *m) {
    if (m->train_exec) cudaGraphExecDestroy(m->train_exec);
    if (m->train_graph) cudaGraphDestroy(m->train_graph);
    m->train_exec = nullptr;
    m->train_graph = nullptr;
    m->train_n = 0;
}

// Capture the training step for batch size n and find the nodes whose
// arguments change between steps (the two standardisations, AdamW).
cudaError_t capture_train(turret_mlp *m, const float *x, const float *y, int n, const turret_adamw *opt) {
    drop_train_graph(m);
    cudaGraph_t gr;
    cudaError_t e = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    e = enqueue_train(m, x, y, n, opt, 1.0f, 1.0f);
    cudaError_t e2 = cudaStreamEndCapture(m->stream, &gr);
    if (e != cudaSuccess) {
        if (e2 == cudaSuccess) cudaGraphDestroy(gr);
        return e;
    }
    if (e2 != cudaSuccess) return e2;
    size_t nn = 0;
    m->node_x = m->node_y = m->node_adam = nullptr;
    e = cudaGraphGetNodes(gr, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess) e = cudaGraphGetNodes(gr, nodes.data(), &nn);
    for (size_t k = 0; k < nn && e == cudaSuccess; ++k) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[k], &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if ((e = cudaGraphKernelNodeGetParams(nodes[k], &kp)) != cudaSuccess) break;
        if (kp.func == (void *)k_adamw) m->node_adam = nodes[k];
        if (kp.func == (void *)k_standardise) {
            const int d = *static_cast<const int *>(kp.kernelParams[2]);
            (d == MLP_IN ? m->node_x : m->node_y) = nodes[k];
        }
    }
    if (e == cudaSuccess && (!m->node_x || !m->node_y || !m->node_adam)) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&m->train_exec, gr, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(gr);
        m->train_exec = nullptr;
        return e;
    }
    m->train_graph = gr;
    m->train_n = n;
    return cudaSuccess;
}

// Replay the captured step with this step's inputs and optimiser scalars.
cudaError_t replay_train(turret_mlp *m, const float *x, const float *y, int n, const turret_adamw *opt, float bc1,
                         float bc2) {
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof kp);
    int d = MLP_IN;
    const float *mean = m->norm, *stdv = m->norm + MLP_IN;
    float *outp = m->X0;
    void *args_x[6] = {&x, &n, &d, &mean, &stdv, &outp};
    kp.func = (void *)k_standardise;
    kp.gridDim = dim3((n * MLP_IN + 255) / 256);
    kp.blockDim = dim3(256);
    kp.kernelParams = args_x;
    cudaError_t e = cudaGraphExecKernelNodeSetParams(m->train_exec, m->node_x, &kp);
    if (e != cudaSuccess) return e;
    int dy = MLP_OUT;
    const float *meany = m->norm + 2 * MLP_IN, *stdy = m->norm + 2 * MLP_IN + MLP_OUT;
    float *outy = m->T;
    void *args_y[6] = {&y, &n, &dy, &meany, &stdy, &outy};
    kp.gridDim = dim3((n * MLP_OUT + 255) / 256);
    kp.kernelParams = args_y;
    if ((e = cudaGraphExecKernelNodeSetParams(m->train_exec, m->node_y, &kp)) != cudaSuccess) return e;
    float lr = opt->lr, b1 = opt->beta1, b2 = opt->beta2, eps = opt->eps, wd = opt->weight_decay;
    void *args_a[11] = {&m->P, &m->G, &m->Mm, &m->Vv, &lr, &b1, &b2, &eps, &wd, &bc1, &bc2};
    kp.func = (void *)k_adamw;
    kp.gridDim = dim3((MLP_NPARAM + 255) / 256);
    kp.kernelParams = args_a;
    if ((e = cudaGraphExecKernelNodeSetParams(m->train_exec, m->node_adam, &kp)) != cudaSuccess) return e;
    return cudaGraphLaunch(m->train_exec, m->stream);
}
}  // namespace

extern "C" turret_status mlp_train_step(turret_mlp *m, const float *x, const float *y, int32_t n,
                                        const turret_adamw *opt, float *loss) {
    if (!m || !x || !y || !opt) return mfail(m, TURRET_EINVAL, "NULL argument");
    if (n < 1 || n > m->cap) return mfail(m, TURRET_EINVAL, "batch outside 1..capacity");
    if (!(opt->lr >= 0.0f) || !(opt->beta1 >= 0.0f && opt->beta1 < 1.0f) || !(opt->beta2 >= 0.0f && opt->beta2 < 1.0f) ||
        !(opt->eps > 0.0f) || !(opt->weight_decay >= 0.0f))
        return mfail(m, TURRET_EINVAL, "invalid optimiser settings");
    m->adam_step += 1;
    const float bc1 = (float)(1.0 - pow((double)opt->beta1, (double)m->adam_step));
    const float bc2 = (float)(1.0 - pow((double)opt->beta2, (double)m->adam_step));
    if (m->stream) {
        // a graph replay per step (the captured step has ~25 kernels)
        if (m->train_n != n) MK(capture_train(m, x, y, n, opt), "training graph capture");
        MK(replay_train(m, x, y, n, opt, bc1, bc2), "training graph launch");
    } else {
        MK(enqueue_train(m, x, y, n, opt, bc1, bc2), "training step");
    }
    if (loss) {
        double L = 0.0;
        MK(cudaMemcpyAsync(&L, m->loss, 8, cudaMemcpyDeviceToHost, m->stream), "loss");
        MK(cudaStreamSynchronize(m->stream), "loss sync");
        *loss = (float)L;
    }
    return TURRET_OK;
}

extern "C" turret_status mlp_destroy(turret_mlp *m) {
    if (!m) return TURRET_EINVAL;
    if (m->stream) cudaStreamSynchronize(m->stream);
    drop_train_graph(m);
    delete m;
    return TURRET_OK;
}

extern "C" const char *mlp_last_error(const turret_mlp *m) { return m ? m->err.c_str() : g_mlp_err.c_str(); }

extern "C" turret_status mlp_build_samples(const double *log, int64_t n_records, float *x, float *y, int32_t *bad,
                                           void *stream) {
    if (!log || !x || !y || !bad || n_records < 5) return TURRET_EINVAL;
    const long long ns = n_records - 4;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(bad, 0, sizeof(int32_t), s) != cudaSuccess) return TURRET_ECUDA;
    k_build_samples<<<(unsigned)((ns + 127) / 128), 128, 0, s>>>(log, ns, x, y, bad);
    return cudaGetLastError() == cudaSuccess ? TURRET_OK : TURRET_ECUDA;
}

// Device view of a network, for the step's predictor.
const MlpDev *mlp_device_view(const turret_mlp *m) { return m ? &m->dev : nullptr; }
