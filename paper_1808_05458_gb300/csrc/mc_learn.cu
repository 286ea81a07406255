// mc_learn.cu -- a learned bound proposer: a small message-passing network
// scores every vertex, and the best sweep cut over the scores (an exact
// integer cut of G) is offered as an upper bound on lambda.  The paper has no
// learned component; the solver only uses the bound when it is below the
// bound it already has, so lambda never depends on the network.
//
// Network (hidden H = 64, F = 8 input features, 3 layers):
//   x_v   = [1, log1p(d_v)/8, log1p(a_v)/8, min(d_v/delta - 1, 8)/8,
//            log1p(mean neighbour degree)/8, log1p(min neighbour degree)/8,
//            q1_v, q2_v]     (d weighted degree, a arcs; q = two seeded
//            random vectors in [-1, 1) after kSmooth steps of the lazy random
//            walk s <- (s + D^-1 A s) / 2, centred by their degree-weighted
//            mean and scaled to largest magnitude 1: the two sides of a
//            sparse cut drift apart under the walk while each side evens out)
//   h0    = ReLU(x W_in + b_in)
//   g_l   = D^-1 A h_l                (mean over neighbours, weighted)
//   h_l+1 = ReLU([h_l, g_l] W_l + b_l)     W_l: 128 x 64, l = 0, 1, 2
//   s_v   = h_3 w_out + b_out         (logit)
// W_l and the activations h, g are BF16 (rounded to nearest even); every sum
// is FP32.  The dense transforms run on the tensor cores (mma.sync m16n8k16,
// BF16 in, FP32 accumulate): they move 384 B and do 16 kflop per row, far
// under the tensor roofline, so a layer is bound by the neighbour gathers
// (128 B per arc).
// Loss: the side of a cut is only defined up to polarity, so per graph
//   L = min(BCE(p, y), BCE(p, 1 - y)) / n,  p = sigmoid(s).
// Training: backward in FP32 with dZ rounded to BF16 where it enters the
// dense products (dX = dZ W^T and dW = X^T dZ, both on the tensor cores; the
// bias gradients sum dZ in FP32), Adam on FP32 master weights.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "mc_internal.cuh"

namespace mc {

constexpr int kF = 8, kH = 64, kL = 3, kK = 2 * kH;
constexpr int kSmooth = 32;   // lazy random-walk steps of the smoothed features
constexpr int kRedBlocks = 256;
// parameter offsets (floats)
constexpr int kPWin = 0, kPBin = kPWin + kF * kH;
constexpr int kPW0 = kPBin + kH;                     // layer l: W (kK x kH) then b (kH)
constexpr int kPLayer = kK * kH + kH;
constexpr int kPWout = kPW0 + kL * kPLayer, kPBout = kPWout + kH;
constexpr int kPTotal = kPBout + 1;

namespace {

__device__ __forceinline__ float u01s(u64 h) { return (float)((h >> 40) & 0xFFFFFF) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------- features --
// the two seeded random vectors of the smoothed features.  The walk runs in
// double precision: once the walk has evened a side out, centring leaves a
// small remainder of a large common value, which single precision would not
// resolve.
__global__ void k_rand_init(int n, u64 seed, double2 *__restrict__ S) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const u64 h = splitmix64(seed ^ splitmix64((u64)(unsigned)v));
        S[v] = make_double2(2.0 * (double)u01s(h) - 1.0, 2.0 * (double)u01s(splitmix64(h)) - 1.0);
    }
}

// one lazy random-walk step: out = (in + D^-1 A in) / 2 (a vertex without
// arcs keeps in / 2); one warp per vertex
__global__ void k_smooth(DevGraph g, const double2 *__restrict__ in, double2 *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < g.n; v += nw) {
        double sx = 0.0, sy = 0.0;
        for (int i = g.rp[v] + lane; i < g.rp[v + 1]; i += 32) {
            const int2 e = g.adj[i];
            const double2 x = in[e.x];
            sx += (double)e.y * x.x;
            sy += (double)e.y * x.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (lane == 0) {
            const double d = (double)g.deg[v];
            const double2 x = in[v];
            out[v] = d > 0 ? make_double2(0.5 * (x.x + sx / d), 0.5 * (x.y + sy / d))
                           : make_double2(0.5 * x.x, 0.5 * x.y);
        }
    }
}

// degree-weighted sums of the smoothed vectors: per-block partials (sum d sx,
// sum d sy, sum d) in double, fixed grid, then one block adds them in order
__global__ void __launch_bounds__(256) k_center_partial(DevGraph g, const double2 *__restrict__ S,
                                                        double *__restrict__ part) {
    __shared__ double sh[3][8];
    double a = 0, b = 0, c = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += gridDim.x * blockDim.x) {
        const double d = (double)g.deg[v];
        a += d * S[v].x;
        b += d * S[v].y;
        c += d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = a; sh[1][threadIdx.x >> 5] = b; sh[2][threadIdx.x >> 5] = c; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0;
        for (int k = 0; k < 8; ++k) t += sh[threadIdx.x][k];
        part[blockIdx.x * 3 + threadIdx.x] = t;
    }
}

// cs[0..1] = the degree-weighted means; the largest magnitudes of the
// centred vectors go to cs[2..3] (as double bits, via integer maxima of
// non-negative doubles) in k_maxabs
__global__ void k_center_final(const double *__restrict__ part, int nb, double *cs) {
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int k = 0; k < nb; ++k) { a += part[3 * k]; b += part[3 * k + 1]; c += part[3 * k + 2]; }
        cs[0] = c > 0 ? a / c : 0.0;
        cs[1] = c > 0 ? b / c : 0.0;
        cs[2] = 0.0;
        cs[3] = 0.0;
    }
}

__global__ void k_maxabs(int n, const double2 *__restrict__ S, double *cs) {
    double mx = 0.0, my = 0.0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        mx = fmax(mx, fabs(S[v].x - cs[0]));
        my = fmax(my, fabs(S[v].y - cs[1]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned long long *>(cs + 2), (unsigned long long)__double_as_longlong(mx));
        atomicMax(reinterpret_cast<unsigned long long *>(cs + 3), (unsigned long long)__double_as_longlong(my));
    }
}

__global__ void k_features(DevGraph g, long long delta, const double2 *__restrict__ Sm, const double *__restrict__ cs,
                           const float *__restrict__ P, float *__restrict__ X, __nv_bfloat16 *__restrict__ H0,
                           float *__restrict__ Z0) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < g.n; v += nw) {
        const int a0 = g.rp[v], a1 = g.rp[v + 1];
        long long sum = 0;  // exact; the features themselves are float
        long long mn = LLONG_MAX;
        for (int i = a0 + lane; i < a1; i += 32) {
            const long long du = g.deg[g.adj[i].x];
            sum += du;
            mn = du < mn ? du : mn;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            const long long om = __shfl_xor_sync(0xffffffffu, mn, o);
            mn = om < mn ? om : mn;
        }
        const int a = a1 - a0;
        const float d = (float)g.deg[v];
        float x[kF];
        x[0] = 1.f;
        x[1] = log1pf(d) / 8.f;
        x[2] = log1pf((float)a) / 8.f;
        const float rel = delta > 0 ? d / (float)delta - 1.f : 0.f;
        x[3] = (rel < 8.f ? rel : 8.f) / 8.f;
        x[4] = log1pf(a > 0 ? (float)sum / (float)a : 0.f) / 8.f;
        x[5] = log1pf(a > 0 ? (float)mn : 0.f) / 8.f;
        const double2 q = Sm[v];
        x[6] = (float)(cs[2] > 0.0 ? (q.x - cs[0]) / cs[2] : q.x - cs[0]);
        x[7] = (float)(cs[3] > 0.0 ? (q.y - cs[1]) / cs[3] : q.y - cs[1]);
        if (lane < kF) X[(size_t)v * kF + lane] = x[lane];
        // h0 = ReLU(x W_in + b_in): lane j computes features j and j + 32
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int j = lane + 32 * t;
            float z = P[kPBin + j];
#pragma unroll
            for (int f = 0; f < kF; ++f) z += x[f] * P[kPWin + f * kH + j];
            Z0[(size_t)v * kH + j] = z;
            H0[(size_t)v * kH + j] = __float2bfloat16(z > 0.f ? z : 0.f);
        }
    }
}

// ----------------------------------------------------------- aggregation --
// G[v] = sum_u (w_uv / d_v) H[u]  (forward);  one warp per vertex, lane owns
// features 2*lane, 2*lane+1 (one 128 B row per neighbour per warp)
__global__ void k_spmm_fwd(DevGraph g, const __nv_bfloat16 *__restrict__ H, __nv_bfloat16 *__restrict__ G) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const __nv_bfloat162 *H2 = reinterpret_cast<const __nv_bfloat162 *>(H);
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < g.n; v += nw) {
        const int a0 = g.rp[v], a1 = g.rp[v + 1];
        float s0 = 0.f, s1 = 0.f;
        for (int i = a0; i < a1; ++i) {
            const int2 e = g.adj[i];
            const float2 hv = __bfloat1622float2(H2[(size_t)e.x * (kH / 2) + lane]);
            s0 += (float)e.y * hv.x;
            s1 += (float)e.y * hv.y;
        }
        const float inv = g.deg[v] > 0 ? 1.f / (float)g.deg[v] : 0.f;
        reinterpret_cast<__nv_bfloat162 *>(G)[(size_t)v * (kH / 2) + lane] =
            __floats2bfloat162_rn(s0 * inv, s1 * inv);
    }
}

// dH[u] += sum_v (w_uv / d_v) dG[v]  (transpose; the graph is symmetric)
__global__ void k_spmm_bwd(DevGraph g, const float *__restrict__ dG, float *__restrict__ dH) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < g.n; u += nw) {
        const int a0 = g.rp[u], a1 = g.rp[u + 1];
        float s0 = 0.f, s1 = 0.f;
        for (int i = a0; i < a1; ++i) {
            const int2 e = g.adj[i];
            const float c = (float)e.y / (float)g.deg[e.x];
            const float2 d = reinterpret_cast<const float2 *>(dG)[(size_t)e.x * (kH / 2) + lane];
            s0 += c * d.x;
            s1 += c * d.y;
        }
        float2 *o = reinterpret_cast<float2 *>(dH) + (size_t)u * (kH / 2) + lane;
        float2 cur = *o;
        cur.x += s0;
        cur.y += s1;
        *o = cur;
    }
}

// --------------------------------------------------------- tensor cores --
__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(unsigned &r0, unsigned &r1, const void *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(a));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Y[rows x N] = A[rows x K] * B[K x N] (+ bias) with A given as up to two
// BF16 row blocks of K/2 columns (A = [A1, A2]) or one of K columns, and B as
// BT[N][K] BF16 (n-major, k contiguous).  64 rows per block of 4 warps.
// mode 0: store Z (fp32) and ReLU(Z) as BF16 into Ybf;  mode 1: store Y fp32.
template <int K, int N>
__global__ void __launch_bounds__(128)
k_gemm(const __nv_bfloat16 *__restrict__ A1, const __nv_bfloat16 *__restrict__ A2, int n_rows,
       const __nv_bfloat16 *__restrict__ BT, const float *__restrict__ bias, float *__restrict__ Zout,
       __nv_bfloat16 *__restrict__ Ybf, int mode) {
    constexpr int KP = K + 8;  // padded row (bf16) against ldmatrix bank conflicts
    __shared__ __align__(16) __nv_bfloat16 sA[64 * KP];
    __shared__ __align__(16) __nv_bfloat16 sB[N * KP];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // B^T to shared memory once per block
    for (int i = tid; i < N * K / 8; i += 128) {
        const int r = i / (K / 8), c8 = i % (K / 8);
        *reinterpret_cast<uint4 *>(&sB[r * KP + c8 * 8]) = reinterpret_cast<const uint4 *>(BT)[(size_t)r * (K / 8) + c8];
    }
    for (int r0 = blockIdx.x * 64; r0 < n_rows; r0 += gridDim.x * 64) {
        __syncthreads();
        // A rows r0..r0+63 (zero past the end)
        for (int i = tid; i < 64 * K / 8; i += 128) {
            const int r = i / (K / 8), c8 = i % (K / 8);
            uint4 val = make_uint4(0, 0, 0, 0);
            if (r0 + r < n_rows) {
                if (A2 == nullptr) {
                    val = reinterpret_cast<const uint4 *>(A1)[(size_t)(r0 + r) * (K / 8) + c8];
                } else if (c8 < K / 16) {
                    val = reinterpret_cast<const uint4 *>(A1)[(size_t)(r0 + r) * (K / 16) + c8];
                } else {
                    val = reinterpret_cast<const uint4 *>(A2)[(size_t)(r0 + r) * (K / 16) + c8 - K / 16];
                }
            }
            *reinterpret_cast<uint4 *>(&sA[r * KP + c8 * 8]) = val;
        }
        __syncthreads();
        float acc[N / 8][4];
#pragma unroll
        for (int t = 0; t < N / 8; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
        const int wr = wid * 16;
#pragma unroll
        for (int k0 = 0; k0 < K; k0 += 16) {
            unsigned a0, a1, a2, a3;
            ldsm_x4(a0, a1, a2, a3, &sA[(wr + (lane & 15)) * KP + k0 + (lane >> 4) * 8]);
#pragma unroll
            for (int t = 0; t < N / 8; ++t) {
                unsigned b0, b1;
                ldsm_x2(b0, b1, &sB[(t * 8 + (lane & 7)) * KP + k0 + ((lane >> 3) & 1) * 8]);
                mma_bf16(acc[t], a0, a1, a2, a3, b0, b1);
            }
        }
        const int rlo = r0 + wr + (lane >> 2), rhi = rlo + 8;
#pragma unroll
        for (int t = 0; t < N / 8; ++t) {
            const int c = t * 8 + (lane & 3) * 2;
            const float b0 = bias ? bias[c] : 0.f, b1 = bias ? bias[c + 1] : 0.f;
            const float z0 = acc[t][0] + b0, z1 = acc[t][1] + b1, z2 = acc[t][2] + b0, z3 = acc[t][3] + b1;
            if (mode == 0) {
                if (rlo < n_rows) {
                    Zout[(size_t)rlo * N + c] = z0;
                    Zout[(size_t)rlo * N + c + 1] = z1;
                    reinterpret_cast<__nv_bfloat162 *>(Ybf)[((size_t)rlo * N + c) / 2] =
                        __floats2bfloat162_rn(z0 > 0.f ? z0 : 0.f, z1 > 0.f ? z1 : 0.f);
                }
                if (rhi < n_rows) {
                    Zout[(size_t)rhi * N + c] = z2;
                    Zout[(size_t)rhi * N + c + 1] = z3;
                    reinterpret_cast<__nv_bfloat162 *>(Ybf)[((size_t)rhi * N + c) / 2] =
                        __floats2bfloat162_rn(z2 > 0.f ? z2 : 0.f, z3 > 0.f ? z3 : 0.f);
                }
            } else {
                if (rlo < n_rows) { Zout[(size_t)rlo * N + c] = z0; Zout[(size_t)rlo * N + c + 1] = z1; }
                if (rhi < n_rows) { Zout[(size_t)rhi * N + c] = z2; Zout[(size_t)rhi * N + c + 1] = z3; }
            }
        }
    }
}

// logits s = h3 . w_out + b_out
__global__ void k_head(const __nv_bfloat16 *__restrict__ H, int n, const float *__restrict__ P, float *__restrict__ S) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
        const float2 h = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(H)[(size_t)v * (kH / 2) + lane]);
        float s = h.x * P[kPWout + 2 * lane] + h.y * P[kPWout + 2 * lane + 1];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) S[v] = s + P[kPBout];
    }
}

__device__ __forceinline__ double bce(double p, int y) {
    const double eps = 1e-7;
    p = p < eps ? eps : (p > 1 - eps ? 1 - eps : p);
    return y ? -log(p) : -log(1 - p);
}

// both polarity losses (sums) into acc[0], acc[1]
__global__ void k_loss(const float *__restrict__ S, const unsigned *__restrict__ bits, int n, double *acc) {
    double l0 = 0, l1 = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double p = 1.0 / (1.0 + exp(-(double)S[v]));
        const int y = (bits[v >> 5] >> (v & 31)) & 1;
        l0 += bce(p, y);
        l1 += bce(p, 1 - y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l0 += __shfl_xor_sync(0xffffffffu, l0, o);
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    }
    if ((threadIdx.x & 31) == 0) { atomicAdd(&acc[0], l0); atomicAdd(&acc[1], l1); }
}

// dS = (p - y*) / n with the better polarity; dH3 = dS w_out; head grads
__global__ void k_head_bwd(const float *__restrict__ S, const unsigned *__restrict__ bits, int n, const double *acc,
                           const __nv_bfloat16 *__restrict__ H, const float *__restrict__ P, float *__restrict__ dH,
                           float *__restrict__ grad) {
    const int flip = acc[1] < acc[0];
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    float gw0 = 0.f, gw1 = 0.f, gb = 0.f;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
        const float p = 1.f / (1.f + expf(-S[v]));
        const int y = ((bits[v >> 5] >> (v & 31)) & 1) ^ flip;
        const float ds = (p - (float)y) / (float)n;
        const float2 h = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(H)[(size_t)v * (kH / 2) + lane]);
        gw0 += ds * h.x;
        gw1 += ds * h.y;
        gb += lane == 0 ? ds : 0.f;
        reinterpret_cast<float2 *>(dH)[(size_t)v * (kH / 2) + lane] =
            make_float2(ds * P[kPWout + 2 * lane], ds * P[kPWout + 2 * lane + 1]);
    }
    atomicAdd(&grad[kPWout + 2 * lane], gw0);
    atomicAdd(&grad[kPWout + 2 * lane + 1], gw1);
    if (lane == 0) atomicAdd(&grad[kPBout], gb);
}

// dZ = dH * (Z > 0) as BF16 (input of dX = dZ W^T) and kept in fp32 in dH
__global__ void k_relu_bwd(float *__restrict__ dH, const float *__restrict__ Z, __nv_bfloat16 *__restrict__ dZbf,
                           long long count) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        const float d = Z[i] > 0.f ? dH[i] : 0.f;
        dH[i] = d;
        dZbf[i] = __float2bfloat16(d);
    }
}

// dW[128 x 64] += X^T bf16(dZ) on the tensor cores and db[64] += the column
// sums of dZ (FP32), with X = [A1, A2] (n x 64 BF16 each).  Tiles of 16
// vertices pass through shared memory; ldmatrix.trans turns the row-major
// tiles into the A (X^T) and B (dZ) fragments of mma.m16n8k16.  Warp w keeps
// rows 32w..32w+31 of dW in registers and adds them into dW at the end.
__global__ void __launch_bounds__(128)
k_wgrad_tc(const __nv_bfloat16 *__restrict__ A1, const __nv_bfloat16 *__restrict__ A2,
           const __nv_bfloat16 *__restrict__ dZb, const float *__restrict__ dZ, int n, float *__restrict__ dW,
           float *__restrict__ db) {
    constexpr int XP = kK + 8, ZP = kH + 8;  // padded rows: 272 B and 144 B, both 16 B multiples
    __shared__ __align__(16) __nv_bfloat16 sX[16 * XP];
    __shared__ __align__(16) __nv_bfloat16 sZ[16 * ZP];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float acc[2][8][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
    float bsum = 0.f;
    const uint4 *X1 = reinterpret_cast<const uint4 *>(A1), *X2 = reinterpret_cast<const uint4 *>(A2);
    const uint4 *Zb = reinterpret_cast<const uint4 *>(dZb);
    for (int v0 = blockIdx.x * 16; v0 < n; v0 += gridDim.x * 16) {
        __syncthreads();
        for (int i = tid; i < 16 * 16; i += 128) {
            const int r = i >> 4, c8 = i & 15;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (v0 + r < n) val = c8 < 8 ? X1[(size_t)(v0 + r) * 8 + c8] : X2[(size_t)(v0 + r) * 8 + c8 - 8];
            *reinterpret_cast<uint4 *>(&sX[r * XP + c8 * 8]) = val;
        }
        {
            const int r = tid >> 3, c8 = tid & 7;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (v0 + r < n) val = Zb[(size_t)(v0 + r) * 8 + c8];
            *reinterpret_cast<uint4 *>(&sZ[r * ZP + c8 * 8]) = val;
        }
        if (tid < kH)
            for (int r = 0; r < 16 && v0 + r < n; ++r) bsum += dZ[(size_t)(v0 + r) * kH + tid];
        __syncthreads();
        unsigned a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int m0 = wid * 32 + mt * 16;
            ldsm_x4_t(a[mt][0], a[mt][1], a[mt][2], a[mt][3],
                      &sX[((lane & 7) + 8 * (lane >> 4)) * XP + m0 + 8 * ((lane >> 3) & 1)]);
        }
#pragma unroll
        for (int nt2 = 0; nt2 < 4; ++nt2) {
            const int n0 = nt2 * 16;
            unsigned b0, b1, b2, b3;
            ldsm_x4_t(b0, b1, b2, b3, &sZ[((lane & 7) + 8 * ((lane >> 3) & 1)) * ZP + n0 + 8 * (lane >> 4)]);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                mma_bf16(acc[mt][2 * nt2], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                mma_bf16(acc[mt][2 * nt2 + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
            }
        }
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int m = wid * 32 + mt * 16 + g, c = nt * 8 + 2 * t;
            atomicAdd(&dW[m * kH + c], acc[mt][nt][0]);
            atomicAdd(&dW[m * kH + c + 1], acc[mt][nt][1]);
            atomicAdd(&dW[(m + 8) * kH + c], acc[mt][nt][2]);
            atomicAdd(&dW[(m + 8) * kH + c + 1], acc[mt][nt][3]);
        }
    if (tid < kH) atomicAdd(&db[tid], bsum);
}

// dW[K x N] += X^T dZ, db += column sums of dZ, on CUDA cores, for the input
// layer (X = the n x 8 FP32 features)
template <int K>
__global__ void __launch_bounds__(256)
k_wgrad(const __nv_bfloat16 *__restrict__ A1, const __nv_bfloat16 *__restrict__ A2, const float *__restrict__ Xf,
        const float *__restrict__ dZ, int n, float *__restrict__ dW, float *__restrict__ db) {
    // thread t owns output column j = t % 64 and rows k = t / 64 + 4 i
    const int t = threadIdx.x, j = t & 63, k0 = t >> 6;
    constexpr int KR = K / 4;
    float acc[KR];
#pragma unroll
    for (int i = 0; i < KR; ++i) acc[i] = 0.f;
    float bsum = 0.f;
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const float dz = dZ[(size_t)v * kH + j];
        if (k0 == 0) bsum += dz;
#pragma unroll
        for (int i = 0; i < KR; ++i) {
            const int k = k0 + 4 * i;
            float x;
            if (Xf) x = Xf[(size_t)v * K + k];
            else if (A2 == nullptr) x = __bfloat162float(A1[(size_t)v * K + k]);
            else x = k < K / 2 ? __bfloat162float(A1[(size_t)v * (K / 2) + k]) : __bfloat162float(A2[(size_t)v * (K / 2) + k - K / 2]);
            acc[i] += x * dz;
        }
    }
#pragma unroll
    for (int i = 0; i < KR; ++i) atomicAdd(&dW[(k0 + 4 * i) * kH + j], acc[i]);
    if (k0 == 0) atomicAdd(&db[j], bsum);
}

__global__ void k_adam(float *P, const float *__restrict__ G, float *M, float *V, int np, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M[i] + (1.f - b1) * g, v = b2 * V[i] + (1.f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// BF16 copies of the dense weights: WT[l] = W_l^T (64 x 128, k contiguous)
// for the forward, W[l] (128 x 64) for dX = dZ W^T
__global__ void k_cast_weights(const float *__restrict__ P, __nv_bfloat16 *WT, __nv_bfloat16 *Wn) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kL * kK * kH; i += gridDim.x * blockDim.x) {
        const int l = i / (kK * kH), r = i % (kK * kH), k = r / kH, j = r % kH;
        const float w = P[kPW0 + l * kPLayer + k * kH + j];
        WT[(size_t)l * kK * kH + j * kK + k] = __float2bfloat16(w);
        Wn[(size_t)l * kK * kH + k * kH + j] = __float2bfloat16(w);
    }
}

// dX (fp32, n x 128) -> dH_direct (cols 0..63, added) and dG (cols 64..127)
__global__ void k_split_dx(const float *__restrict__ dX, int n, float *__restrict__ dH, float *__restrict__ dG) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)n * kK;
         i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / kK;
        const int c = (int)(i % kK);
        if (c < kH) dH[v * kH + c] = dX[i];
        else dG[v * kH + c - kH] = dX[i];
    }
}

// ---------------------------------------------------------- sweep cut --
// rank[v] = position of v in ascending score order (ties by vertex id)
__global__ void k_score_keys(const float *__restrict__ S, int n, u64 *keys, int *vals) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        unsigned b = __float_as_uint(S[v]);
        b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // order-preserving
        keys[v] = (u64)b;  // the stable sort keeps equal scores in vertex order
        vals[v] = v;
    }
}
__global__ void k_rank(const int *__restrict__ order, int n, int *rank) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) rank[order[i]] = i;
}
// term[rank v] = d_v - 2 * (weight from v to lower-ranked vertices)
__global__ void k_sweep_terms(DevGraph g, const int *__restrict__ rank, long long *term) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += gridDim.x * blockDim.x) {
        long long t = g.deg[v];
        const int rv = rank[v];
        for (int i = g.rp[v]; i < g.rp[v + 1]; ++i) {
            const int2 e = g.adj[i];
            if (rank[e.x] < rv) t -= 2LL * e.y;
        }
        term[rv] = t;
    }
}
// Minimum over the prefix sums P(k) = term[0] + ... + term[k-1], k = 1..n-1
// (the cut between the k lowest-ranked vertices and the rest), smallest k
// on ties.  Tiles of kSwTile terms: tile sums, one scan of the tile sums,
// per-tile minima, one final reduction.
constexpr int kSwThreads = 256, kSwItems = 8, kSwTile = kSwThreads * kSwItems;

__device__ __forceinline__ long long block_excl_scan_ll(long long v, long long *total) {
    __shared__ long long ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const long long x = lane < nwarp ? ws[lane] : 0;
        long long xs = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, xs, o);
            if (lane >= o) xs += t;
        }
        if (lane < nwarp) ws[lane] = xs - x;
        if (lane == nwarp - 1) *total = xs;
    }
    __syncthreads();
    const long long r = ws[wid] + inc - v;
    __syncthreads();
    return r;
}

__device__ __forceinline__ void better_cut(long long &mb, int &mk, long long ob, int ok) {
    if (ob < mb || (ob == mb && ok < mk)) { mb = ob; mk = ok; }
}

__device__ void block_min_cut(long long &mb, int &mk) {
    __shared__ long long wb[32];
    __shared__ int wk[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        better_cut(mb, mk, __shfl_xor_sync(0xffffffffu, mb, o), __shfl_xor_sync(0xffffffffu, mk, o));
    if (lane == 0) { wb[wid] = mb; wk[wid] = mk; }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) better_cut(mb, mk, wb[k], wk[k]);
    __syncthreads();
}

__global__ void __launch_bounds__(kSwThreads) k_sw_tile_sum(const long long *__restrict__ term, int n,
                                                            long long *tsum) {
    __shared__ long long total;
    const long long base = (long long)blockIdx.x * kSwTile + (long long)threadIdx.x * kSwItems;
    long long v = 0;
#pragma unroll
    for (int k = 0; k < kSwItems; ++k)
        if (base + k < n) v += term[base + k];
    block_excl_scan_ll(v, &total);
    if (threadIdx.x == 0) tsum[blockIdx.x] = total;
}

// exclusive scan of the T tile sums in place (one block)
__global__ void k_sw_tile_scan(long long *tsum, int T) {
    __shared__ long long total;
    long long carry = 0;
    for (int base = 0; base < T; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const long long v = i < T ? tsum[i] : 0;
        const long long ex = block_excl_scan_ll(v, &total);
        if (i < T) tsum[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSwThreads) k_sw_tile_min(const long long *__restrict__ term, int n,
                                                            const long long *__restrict__ toff,
                                                            long long *bmin, int *bk) {
    __shared__ long long total;
    const long long base = (long long)blockIdx.x * kSwTile + (long long)threadIdx.x * kSwItems;
    long long t[kSwItems];
    long long v = 0;
#pragma unroll
    for (int k = 0; k < kSwItems; ++k) {
        t[k] = base + k < n ? term[base + k] : 0;
        v += t[k];
    }
    long long pre = toff[blockIdx.x] + block_excl_scan_ll(v, &total);
    long long mb = LLONG_MAX;
    int mk = INT_MAX;
#pragma unroll
    for (int k = 0; k < kSwItems; ++k) {
        pre += t[k];  // cut of the first i + 1 vertices
        const long long i = base + k;
        if (i < n - 1) better_cut(mb, mk, pre, (int)(i + 1));
    }
    block_min_cut(mb, mk);
    if (threadIdx.x == 0) { bmin[blockIdx.x] = mb; bk[blockIdx.x] = mk; }
}

__global__ void k_sw_final(const long long *__restrict__ bmin, const int *__restrict__ bk, int T,
                           long long *best, int *best_k) {
    long long mb = LLONG_MAX;
    int mk = INT_MAX;
    for (int i = threadIdx.x; i < T; i += blockDim.x) better_cut(mb, mk, bmin[i], bk[i]);
    block_min_cut(mb, mk);
    if (threadIdx.x == 0) {
        *best = mb;
        *best_k = mk == INT_MAX ? 0 : mk;
    }
}

}  // namespace

// ------------------------------------------------------------- host side --
struct Proposer {
    int n_cap = 0;
    float *P = nullptr, *M = nullptr, *V = nullptr, *grad = nullptr;
    __nv_bfloat16 *WT = nullptr, *Wn = nullptr;
    float *X = nullptr, *Z = nullptr, *S = nullptr, *dH = nullptr, *dG = nullptr, *dX = nullptr;
    double2 *Sm0 = nullptr, *Sm1 = nullptr; // smoothed-feature ping-pong
    double *red = nullptr;                  // centring partials
    double *cs = nullptr;                   // means and largest magnitudes
    __nv_bfloat16 *Hb = nullptr, *Gb = nullptr, *dZb = nullptr;
    double *acc = nullptr;
    int adam_t = 0;
    u64 feat_seed = 0x51ED270B27A4BB1DULL;
};

static int prop_alloc(Proposer &p, int n, cudaStream_t s) {
    if (n <= p.n_cap) return MC_OK;
    void *ps[] = {p.X, p.Z, p.S, p.dH, p.dG, p.dX, p.Hb, p.Gb, p.dZb, p.Sm0, p.Sm1};
    for (void *q : ps) dev_free(q, s);
    const size_t N = (size_t)n;
    MC_TRY(dev_alloc_n(&p.Sm0, N, s));
    MC_TRY(dev_alloc_n(&p.Sm1, N, s));
    MC_TRY(dev_alloc_n(&p.X, N * kF, s));
    MC_TRY(dev_alloc_n(&p.Z, N * kH * (kL + 1), s));
    MC_TRY(dev_alloc_n(&p.S, N, s));
    MC_TRY(dev_alloc_n(&p.dH, N * kH, s));
    MC_TRY(dev_alloc_n(&p.dG, N * kH, s));
    MC_TRY(dev_alloc_n(&p.dX, N * kK, s));
    MC_TRY(dev_alloc_n(&p.Hb, N * kH * (kL + 1), s));
    MC_TRY(dev_alloc_n(&p.Gb, N * kH * kL, s));
    MC_TRY(dev_alloc_n(&p.dZb, N * kH, s));
    p.n_cap = n;
    return MC_OK;
}

int proposer_create(Proposer **out, const float *init) {
    Proposer *p = new Proposer();
    cudaStream_t s = nullptr;
    int rc = MC_OK;
    if ((rc = dev_alloc_n(&p->P, kPTotal, s)) != MC_OK || (rc = dev_alloc_n(&p->M, kPTotal, s)) != MC_OK ||
        (rc = dev_alloc_n(&p->V, kPTotal, s)) != MC_OK || (rc = dev_alloc_n(&p->grad, kPTotal, s)) != MC_OK ||
        (rc = dev_alloc_n(&p->WT, (size_t)kL * kK * kH, s)) != MC_OK ||
        (rc = dev_alloc_n(&p->Wn, (size_t)kL * kK * kH, s)) != MC_OK || (rc = dev_alloc_n(&p->acc, 4, s)) != MC_OK ||
        (rc = dev_alloc_n(&p->red, 3 * kRedBlocks, s)) != MC_OK || (rc = dev_alloc_n(&p->cs, 4, s)) != MC_OK) {
        delete p;
        return rc;
    }
    MC_CUDA(cudaMemcpy(p->P, init, sizeof(float) * kPTotal, cudaMemcpyHostToDevice));
    MC_CUDA(cudaMemset(p->M, 0, sizeof(float) * kPTotal));
    MC_CUDA(cudaMemset(p->V, 0, sizeof(float) * kPTotal));
    *out = p;
    return MC_OK;
}

void proposer_destroy(Proposer *p) {
    if (!p) return;
    void *ps[] = {p->P, p->M, p->V, p->grad, p->WT, p->Wn, p->acc, p->X, p->Z, p->S, p->dH, p->dG, p->dX,
                  p->Hb, p->Gb, p->dZb, p->Sm0, p->Sm1, p->red, p->cs};
    cudaDeviceSynchronize();  // no stream may still use the buffers
    for (void *q : ps) dev_free(q, nullptr);
    delete p;
}

int proposer_set(Proposer *p, const float *w) {
    MC_CUDA(cudaMemcpy(p->P, w, sizeof(float) * kPTotal, cudaMemcpyHostToDevice));
    return MC_OK;
}
int proposer_get(Proposer *p, float *w) {
    MC_CUDA(cudaMemcpy(w, p->P, sizeof(float) * kPTotal, cudaMemcpyDeviceToHost));
    return MC_OK;
}
int proposer_nparams() { return kPTotal; }

static int blocks_for(long long work, int threads) {
    long long b = (work + threads - 1) / threads;
    const long long cap = (long long)num_sms() * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

// forward pass on g; logits in p.S
int proposer_forward(Proposer &p, const DevGraph &g, long long delta, cudaStream_t s) {
    MC_TRY(prop_alloc(p, g.n, s));
    const size_t NH = (size_t)g.n * kH;
    ++::mc::g_launches; k_cast_weights<<<64, 256, 0, s>>>(p.P, p.WT, p.Wn);
    const int wb = blocks_for((long long)g.n * 32, 256);
    const int tb = blocks_for(g.n, 256);
    // smoothed random features: kSmooth lazy-walk steps, centring, scaling
    ++::mc::g_launches; k_rand_init<<<tb, 256, 0, s>>>(g.n, p.feat_seed, p.Sm0);
    double2 *a = p.Sm0, *b = p.Sm1;
    for (int t = 0; t < kSmooth; ++t) {
        ++::mc::g_launches; k_smooth<<<wb, 256, 0, s>>>(g, a, b);
        double2 *tmp = a; a = b; b = tmp;
    }
    ++::mc::g_launches; k_center_partial<<<kRedBlocks, 256, 0, s>>>(g, a, p.red);
    ++::mc::g_launches; k_center_final<<<1, 32, 0, s>>>(p.red, kRedBlocks, p.cs);
    ++::mc::g_launches; k_maxabs<<<tb, 256, 0, s>>>(g.n, a, p.cs);
    ++::mc::g_launches; k_features<<<wb, 256, 0, s>>>(g, delta, a, p.cs, p.P, p.X, p.Hb, p.Z);
    for (int l = 0; l < kL; ++l) {
        const __nv_bfloat16 *H = p.Hb + l * NH;
        __nv_bfloat16 *G = p.Gb + l * NH;
        ++::mc::g_launches; k_spmm_fwd<<<wb, 256, 0, s>>>(g, H, G);
        const int gb = blocks_for(((long long)g.n + 63) / 64 * 128, 128);
        ++::mc::g_launches;
        k_gemm<kK, kH><<<gb, 128, 0, s>>>(H, G, g.n, p.WT + (size_t)l * kK * kH,
                                          p.P + kPW0 + l * kPLayer + kK * kH, p.Z + (l + 1) * NH,
                                          p.Hb + (l + 1) * NH, 0);
    }
    ++::mc::g_launches; k_head<<<wb, 256, 0, s>>>(p.Hb + kL * NH, g.n, p.P, p.S);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

// loss and gradient (p.grad) for labels `bits` (device bitmap); *loss = min
// polarity loss / n
int proposer_backward(Proposer &p, const DevGraph &g, const unsigned *bits, double *loss, cudaStream_t s) {
    const size_t NH = (size_t)g.n * kH;
    MC_CUDA(cudaMemsetAsync(p.acc, 0, sizeof(double) * 4, s));
    MC_CUDA(cudaMemsetAsync(p.grad, 0, sizeof(float) * kPTotal, s));
    const int tb = blocks_for(g.n, 256), wb = blocks_for((long long)g.n * 32, 256);
    ++::mc::g_launches; k_loss<<<tb, 256, 0, s>>>(p.S, bits, g.n, p.acc);
    ++::mc::g_launches; k_head_bwd<<<wb, 256, 0, s>>>(p.S, bits, g.n, p.acc, p.Hb + kL * NH, p.P, p.dH, p.grad);
    for (int l = kL - 1; l >= 0; --l) {
        // dZ_{l+1} = dH_{l+1} * ReLU'
        ++::mc::g_launches; k_relu_bwd<<<blocks_for((long long)NH, 256), 256, 0, s>>>(p.dH, p.Z + (l + 1) * NH, p.dZb, (long long)NH);
        // dW_l (tensor cores), db_l
        ++::mc::g_launches;
        k_wgrad_tc<<<blocks_for(((long long)g.n + 15) / 16 * 128, 128), 128, 0, s>>>(
            p.Hb + l * NH, p.Gb + l * NH, p.dZb, p.dH, g.n, p.grad + kPW0 + l * kPLayer,
            p.grad + kPW0 + l * kPLayer + kK * kH);
        // dX = dZ W_l^T  (n x 128): B^T operand = W_l as (128 x 64) n-major
        const int gb = blocks_for(((long long)g.n + 63) / 64 * 128, 128);
        ++::mc::g_launches;
        k_gemm<kH, kK><<<gb, 128, 0, s>>>(p.dZb, nullptr, g.n, p.Wn + (size_t)l * kK * kH, nullptr, p.dX, nullptr, 1);
        ++::mc::g_launches; k_split_dx<<<blocks_for((long long)g.n * kK, 256), 256, 0, s>>>(p.dX, g.n, p.dH, p.dG);
        ++::mc::g_launches; k_spmm_bwd<<<wb, 256, 0, s>>>(g, p.dG, p.dH);
    }
    // input layer: dZ0 = dH0 * ReLU'(Z0); dW_in = X^T dZ0
    ++::mc::g_launches; k_relu_bwd<<<blocks_for((long long)NH, 256), 256, 0, s>>>(p.dH, p.Z, p.dZb, (long long)NH);
    ++::mc::g_launches;
    k_wgrad<kF><<<num_sms() * 4, 256, 0, s>>>(nullptr, nullptr, p.X, p.dH, g.n, p.grad + kPWin, p.grad + kPBin);
    MC_CUDA(cudaGetLastError());
    double h[4];
    MC_CUDA(cudaMemcpyAsync(h, p.acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    *loss = (h[0] < h[1] ? h[0] : h[1]) / (double)g.n;
    return MC_OK;
}

int proposer_adam(Proposer &p, float lr, cudaStream_t s) {
    ++p.adam_t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)p.adam_t), c2 = 1.f - powf(b2, (float)p.adam_t);
    ++::mc::g_launches; k_adam<<<blocks_for(kPTotal, 256), 256, 0, s>>>(p.P, p.grad, p.M, p.V, kPTotal, lr, b1, b2, 1e-8f, c1, c2);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

int proposer_grad_copy(Proposer &p, float *out) {
    MC_CUDA(cudaMemcpy(out, p.grad, sizeof(float) * kPTotal, cudaMemcpyDeviceToHost));
    return MC_OK;
}
int proposer_logits_copy(Proposer &p, int n, float *out) {
    MC_CUDA(cudaMemcpy(out, p.S, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost));
    return MC_OK;
}

// best sweep cut over the logits of the last forward pass: *cut and, in
// w.T[0..n), the side as 1 for the first k vertices in score order.  Uses the
// radix buffers, w.root (ranks) and w.order (order).
int proposer_sweep(Proposer &p, const DevGraph &g, Work &w, long long *cut, int *k_out, cudaStream_t s) {
    const int n = g.n;
    const int tb = blocks_for(n, 256);
    ++::mc::g_launches; k_score_keys<<<tb, 256, 0, s>>>(p.S, n, w.keysA, w.valsA);
    bool in_b = false;
    MC_TRY(radix_sort_pairs(w.keysA, w.valsA, w.keysB, w.valsB, n, 32, w.radix_tmp, w.scan_tmp, &w.st->err, &in_b, s));
    const int *order = in_b ? w.valsB : w.valsA;
    ++::mc::g_launches; k_rank<<<tb, 256, 0, s>>>(order, n, w.root);
    long long *term = reinterpret_cast<long long *>(in_b ? w.keysA : w.keysB);
    ++::mc::g_launches; k_sweep_terms<<<tb, 256, 0, s>>>(g, w.root, term);
    long long *d_best = reinterpret_cast<long long *>(&w.st->count);
    int *d_k = &w.st->best_len;
    // tile scratch in the sorted-key buffer (free once the ranks are out)
    const int T = (n + kSwTile - 1) / kSwTile;
    long long *tsum = reinterpret_cast<long long *>(in_b ? w.keysB : w.keysA);
    long long *bmin = tsum + T;
    int *bk = reinterpret_cast<int *>(bmin + T);
    ++::mc::g_launches; k_sw_tile_sum<<<T, kSwThreads, 0, s>>>(term, n, tsum);
    ++::mc::g_launches; k_sw_tile_scan<<<1, 1024, 0, s>>>(tsum, T);
    ++::mc::g_launches; k_sw_tile_min<<<T, kSwThreads, 0, s>>>(term, n, tsum, bmin, bk);
    ++::mc::g_launches; k_sw_final<<<1, 1024, 0, s>>>(bmin, bk, T, d_best, d_k);
    MC_CUDA(cudaGetLastError());
    MC_TRY(status_read(w, s));
    *cut = w.h_st->count;
    *k_out = w.h_st->best_len;
    return MC_OK;
}

}  // namespace mc
