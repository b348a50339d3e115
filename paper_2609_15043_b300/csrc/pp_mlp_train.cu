// Training of the proposal network on the device: mixed-precision minibatch
// gradient descent with FP32 master weights, BF16 operands on the tensor
// cores and FP32 accumulation in tensor memory, and an Adam update.
//
// Every product of a step is one tcgen05 GEMM D[M x N] = A[M x K] B[N x K]^T
// with both operands K-major BF16 in global memory and a fused epilogue.  A CTA
// owns a 128 x Nt tile of D (Nt = min(N, 128)) over a range of K (the weight
// gradients, whose K is the batch, split K across CTAs and add their partial
// tiles); K is staged through two shared-memory buffers 64 at a time with
// cp.async, so the next slab loads while the tensor cores work on this one.
// Epilogues:
//   forward, hidden layer l:  H_{l+1} = bf16(relu(H_l W_l^T + b_l)), written
//                             row-major and transposed;
//   forward, output layer:    Y = H_3 W_3^T + b_3 (FP32);
//   weight gradient:          dW_l^T = H_l^T G_l (A = H_l^T, B = G_l^T, both
//                             stored transposed so that K = batch is contiguous);
//   input gradient:           G_{l-1} = (G_l W_l) * [H_l > 0] (B = W_l^T, kept
//                             as a second BF16 copy), FP32 and BF16 copies.
// The loss is the mean squared error over the batch rows and the used outputs;
// G_3 = 2 (Y - T) / (B n_out).  Rows of the batch are padded to a multiple of
// 128 with zero gradient rows, which contribute nothing to any sum.
#include "pp_internal.h"
#include "pp_tc.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace pp {

namespace {

constexpr int kW = 256;          // hidden width and padded input width
constexpr int kOut = 32;         // padded output width
constexpr int kTile = 128;       // rows of D per CTA (MMA M)
constexpr int kSlab = 64;        // K elements staged per round
constexpr int kMaxBatch = 4096;
// parameter block: W0, W1, W2 (256 x 256), W3 (32 x 256), b0, b1, b2 (256), b3 (32)
constexpr int kNW = 3 * kW * kW + kOut * kW;
constexpr int kNP = kNW + 3 * kW + kOut;

__host__ __device__ inline int w_off(int l) { return l * kW * kW; }
__host__ __device__ inline int b_off(int l) { return kNW + l * kW; }
__host__ __device__ inline int rows_of(int l) { return l < 3 ? kW : kOut; }

enum Epi { EPI_HIDDEN = 0, EPI_OUT = 1, EPI_DW = 2, EPI_DX = 3 };

struct GemmArgs {
    const uint16_t* A;
    int lda;                     // M x K, K contiguous (BF16 bits)
    const uint16_t* B;
    int ldb;                     // N x K
    int M, N, K;                 // M % 128 == 0; N in {32, 256}; K % 16 == 0
    int epi;
    const float* bias;           // EPI_HIDDEN, EPI_OUT
    const uint16_t* mask;        // EPI_DX: the layer's input activations [M][N]
    int ldm;
    float* out;                  // EPI_OUT [M][N], EPI_DW [N][M], EPI_DX [M][N]
    int ldo;
    uint16_t* outb;              // row-major BF16 copy (EPI_HIDDEN, EPI_DX)
    int ldob;
    uint16_t* outt;              // transposed BF16 copy [N][M]
    int ldot;
    unsigned* status;
};

constexpr int kNt = 128;         // columns of D per CTA at most

struct GemmSmem {
    uint16_t a[2][kTile * kSlab];   // 2 x 16 KB
    uint16_t b[2][kNt * kSlab];     // 2 x 16 KB
    uint64_t bar[2];
    uint32_t tmem_base;
};

// The dynamic shared memory requested per CTA is larger than two CTAs can
// share, so one CTA per SM holds tensor memory at a time.
constexpr size_t kGemmSmem = 120 * 1024;

__device__ __forceinline__ uint16_t bf16_bits(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// 16 consecutive BF16 values (packed in pairs) to a 32-byte aligned row segment
__device__ __forceinline__ void store_row16(uint16_t* dst, const uint32_t (&pk)[8]) {
    uint4* d = reinterpret_cast<uint4*>(dst);
    d[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    d[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// grid: (M / 128, N / Nt, K splits); K per split a multiple of 16
__global__ void __launch_bounds__(128, 1) tr_gemm(GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    GemmSmem& s = *reinterpret_cast<GemmSmem*>(smraw);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int m0 = blockIdx.x * kTile;
    const int Nt = g.N < kNt ? g.N : kNt;
    const int n0 = blockIdx.y * Nt;
    // K splits on 16-element boundaries (K is a multiple of 16, splits <= K / 16)
    const int units = g.K / 16;
    const int u0 = (int)((long long)units * blockIdx.z / gridDim.z);
    const int u1 = (int)((long long)units * (blockIdx.z + 1) / gridDim.z);
    const int kbeg = 16 * u0, kc = 16 * (u1 - u0);
    const int nslab = (kc + kSlab - 1) / kSlab;
    const uint32_t ncols = Nt <= 32 ? 32u : (uint32_t)kNt;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_addr(
                         &s.tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        tc::mbar_init1(&s.bar[0]);
        tc::mbar_init1(&s.bar[1]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s.tmem_base;

    // slab i of this CTA's K range into buffer `buf` (16-byte pieces: 8 consecutive k of a row)
    auto load_slab = [&](int i, int buf) {
        const int k0 = kbeg + i * kSlab;
        const int kn = min(kSlab, kbeg + kc - k0);
        const int pieces = kn / 8;
        for (int q = t; q < kTile * pieces; q += blockDim.x) {
            const int r = q / pieces, k8 = (q % pieces) * 8;
            cp_async16(reinterpret_cast<char*>(s.a[buf]) + tc::kmajor_off(r, k8, kTile),
                       g.A + (size_t)(m0 + r) * g.lda + k0 + k8);
        }
        for (int q = t; q < Nt * pieces; q += blockDim.x) {
            const int r = q / pieces, k8 = (q % pieces) * 8;
            cp_async16(reinterpret_cast<char*>(s.b[buf]) + tc::kmajor_off(r, k8, Nt),
                       g.B + (size_t)(n0 + r) * g.ldb + k0 + k8);
        }
        cp_async_commit();
    };

    // commits of slab i arrive on bar[i & 1]; each is waited once, in order
    uint32_t phase[2] = {0u, 0u};
    int waited = 0;
    bool ok = true;
    auto wait_slab = [&](int i) -> bool {
        const int b = i & 1;
        const bool done = __syncthreads_and(tc::mbar_wait_bounded(&s.bar[b], phase[b]) ? 1 : 0) != 0;
        if (!done) {
            // the products may still be in flight: one more bounded wait
            // before shared memory or tensor memory is released
            tc::mbar_wait_bounded(&s.bar[b], phase[b]);
            __syncthreads();
        }
        phase[b] ^= 1u;
        waited = i + 1;
        return done;
    };

    load_slab(0, 0);
    int issued = 0;
    for (int i = 0; i < nslab; ++i) {
        const int buf = i & 1;
        if (i + 1 < nslab) {
            // the other buffer held slab i - 1: its products must be complete
            if (i >= 1 && !wait_slab(i - 1)) {
                ok = false;
                break;
            }
            load_slab(i + 1, buf ^ 1);
            cp_async_wait<1>();              // slab i has landed
        } else {
            cp_async_wait<0>();
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int kn = min(kSlab, kbeg + kc - (kbeg + i * kSlab));
            const uint32_t ab = tc::smem_addr(s.a[buf]), bb = tc::smem_addr(s.b[buf]);
            const uint32_t idesc = tc::idesc_bf16(kTile, Nt);
#pragma unroll 1
            for (int ks = 0; ks < kn / 16; ++ks) {
                const uint64_t da = tc::sdesc(ab + (uint32_t)(ks * kTile * 32), 128, 256);
                const uint64_t db = tc::sdesc(bb + (uint32_t)(ks * Nt * 32), 128, 256);
                tc::mma_bf16(tmem, da, db, idesc, (i > 0 || ks > 0) ? 1u : 0u);
            }
            tc::mma_commit(&s.bar[buf]);
        }
        __syncwarp();
        issued = i + 1;
    }
    // every commit is waited before the accumulator is read or the CTA exits
    while (waited < issued) {
        if (!wait_slab(waited)) {
            if (ok && t == 0 && g.status) atomicOr(g.status, (unsigned)PP_ST_TIMEOUT);
            ok = false;
        }
    }
    if (!ok && t == 0 && g.status) atomicOr(g.status, (unsigned)PP_ST_TIMEOUT);
    cp_async_wait<0>();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (ok) {
        // warp w reads TMEM lanes (rows of D) 32w .. 32w + 31
        const int m = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < Nt; c0 += 16) {
            uint32_t v[16];
            tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
            const int n = n0 + c0;
            if (g.epi == EPI_HIDDEN) {
                uint32_t pk[8];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float y = __uint_as_float(v[j]) + g.bias[n + j];
                    const uint16_t hb = bf16_bits(y > 0.f ? y : 0.f);
                    g.outt[(size_t)(n + j) * g.ldot + m] = hb;
                    pk[j >> 1] = (j & 1) ? (pk[j >> 1] | ((uint32_t)hb << 16)) : (uint32_t)hb;
                }
                store_row16(g.outb + (size_t)m * g.ldob + n, pk);
            } else if (g.epi == EPI_OUT) {
                float4* dst = reinterpret_cast<float4*>(g.out + (size_t)m * g.ldo + n);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    dst[j] = make_float4(__uint_as_float(v[4 * j]) + g.bias[n + 4 * j],
                                         __uint_as_float(v[4 * j + 1]) + g.bias[n + 4 * j + 1],
                                         __uint_as_float(v[4 * j + 2]) + g.bias[n + 4 * j + 2],
                                         __uint_as_float(v[4 * j + 3]) + g.bias[n + 4 * j + 3]);
            } else if (g.epi == EPI_DW) {
                // partial sums of the K splits (the output is zeroed first)
#pragma unroll
                for (int j = 0; j < 16; ++j) atomicAdd(&g.out[(size_t)(n + j) * g.ldo + m], __uint_as_float(v[j]));
            } else {
                // the 16 mask activations of this row segment (32 bytes)
                const uint4* mp = reinterpret_cast<const uint4*>(g.mask + (size_t)m * g.ldm + n);
                const uint4 m0v = mp[0], m1v = mp[1];
                const uint32_t mw[8] = {m0v.x, m0v.y, m0v.z, m0v.w, m1v.x, m1v.y, m1v.z, m1v.w};
                uint32_t pk[8];
                float gv[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const uint32_t h = (mw[j >> 1] >> ((j & 1) * 16)) & 0xFFFFu;
                    const bool pass = (h & 0x8000u) == 0 && (h & 0x7FFFu) != 0;   // activation > 0
                    gv[j] = pass ? __uint_as_float(v[j]) : 0.f;
                    const uint16_t gb = bf16_bits(gv[j]);
                    g.outt[(size_t)(n + j) * g.ldot + m] = gb;
                    pk[j >> 1] = (j & 1) ? (pk[j >> 1] | ((uint32_t)gb << 16)) : (uint32_t)gb;
                }
                float4* dst = reinterpret_cast<float4*>(g.out + (size_t)m * g.ldo + n);
#pragma unroll
                for (int j = 0; j < 4; ++j) dst[j] = make_float4(gv[4 * j], gv[4 * j + 1], gv[4 * j + 2], gv[4 * j + 3]);
                store_row16(g.outb + (size_t)m * g.ldob + n, pk);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// batch rows idx[0..B) of the resident set into the layer-0 operands (row-major
// and transposed) and the targets; rows B..Bp are zero
__global__ void tr_gather(const uint16_t* __restrict__ X, const float* __restrict__ Y, const int* __restrict__ idx,
                          int B, int Bp, uint16_t* H0, uint16_t* H0T, float* Yb) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < Bp * kW) {
        // consecutive threads take consecutive rows of one column: the
        // transposed store is coalesced, the row-major one strided
        const int k = q / Bp, r = q % Bp;
        const uint16_t v = r < B ? X[(size_t)idx[r] * kW + k] : (uint16_t)0;
        H0T[(size_t)k * Bp + r] = v;
        H0[(size_t)r * kW + k] = v;
    }
    if (q < Bp * kOut) {
        const int r = q / kOut, o = q % kOut;
        Yb[q] = r < B ? Y[(size_t)idx[r] * kOut + o] : 0.f;
    }
}

// output gradient and the batch's sum of squared errors
__global__ void tr_loss(const float* __restrict__ out, const float* __restrict__ Yb, int B, int Bp, int n_out,
                        float scale, float* G, uint16_t* Gb, uint16_t* GT, double* sse) {
    __shared__ double red[8];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (q < Bp * kOut) {
        const int r = q / kOut, o = q % kOut;
        const float d = (r < B && o < n_out) ? out[q] - Yb[q] : 0.f;
        const float gv = d * scale;
        G[q] = gv;
        const uint16_t b = bf16_bits(gv);
        Gb[q] = b;
        GT[(size_t)o * Bp + r] = b;
        e = (double)d * (double)d;
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        if (s != 0.0) atomicAdd(sse, s);
    }
}

// bias gradient: column sums of the FP32 gradient [Bp][N]; one block per column
__global__ void tr_bias_grad(const float* __restrict__ G, int Bp, int N, float* gb) {
    __shared__ float red[8];
    const int n = blockIdx.x;
    float s = 0.f;
    for (int r = threadIdx.x; r < Bp; r += blockDim.x) s += G[(size_t)r * N + n];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        gb[n] = tot;
    }
}

struct AdamArgs {
    float* P;
    const float* Gr;
    float* m;
    float* v;
    float lr, b1, b2, eps, wd;
    float c1, c2;                // 1 / (1 - b1^t), 1 / (1 - b2^t)
    uint16_t* Wb[4];             // BF16 [out][in]
    uint16_t* WT[4];             // BF16 [in][out]
};

// Adam on every parameter, decoupled weight decay on the weights, then the
// BF16 copies of the weights (both orientations)
__global__ void tr_adam(AdamArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNP) return;
    const float g = a.Gr[i];
    const float m = a.b1 * a.m[i] + (1.0f - a.b1) * g;
    const float v = a.b2 * a.v[i] + (1.0f - a.b2) * g * g;
    a.m[i] = m;
    a.v[i] = v;
    float p = a.P[i] - a.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
    if (i < kNW) {
        p -= a.lr * a.wd * p;
        const int l = i < 3 * kW * kW ? i / (kW * kW) : 3;
        const int e = i - w_off(l);
        const int o = e / kW, k = e % kW;
        const uint16_t b = bf16_bits(p);
        a.Wb[l][e] = b;
        a.WT[l][(size_t)k * rows_of(l) + o] = b;
    }
    a.P[i] = p;
}

// BF16 copies of the master weights (after create)
__global__ void tr_cast(const float* P, AdamArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNW) return;
    const int l = i < 3 * kW * kW ? i / (kW * kW) : 3;
    const int e = i - w_off(l);
    const int o = e / kW, k = e % kW;
    const uint16_t b = bf16_bits(P[i]);
    a.Wb[l][e] = b;
    a.WT[l][(size_t)k * rows_of(l) + o] = b;
}

// standardised features (rows x n_in, FP32) -> BF16 rows of 256; targets -> rows of 32
__global__ void tr_load(const float* __restrict__ x, const float* __restrict__ y, int rows, int n_in, int n_out,
                        uint16_t* X, float* Y) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < (size_t)rows * kW) {
        const size_t r = q / kW;
        const int k = (int)(q % kW);
        X[q] = k < n_in ? bf16_bits(x[r * n_in + k]) : (uint16_t)0;
    }
    if (q < (size_t)rows * kOut) {
        const size_t r = q / kOut;
        const int o = (int)(q % kOut);
        Y[q] = o < n_out ? y[r * n_out + o] : 0.f;
    }
}

}  // namespace

struct Trainer {
    int n_in = 0, n_out = 0, batch = 0, Bp = 0;
    double lr = 0, b1 = 0, b2 = 0, eps = 0, wd = 0;
    long long step = 0;
    int rows = 0;
    uint16_t* X = nullptr;
    float* Y = nullptr;
    int* idx = nullptr;
    int idx_cap = 0;
    float *P = nullptr, *Gr = nullptr, *M = nullptr, *V = nullptr;
    uint16_t* Wb[4] = {};
    uint16_t* WT[4] = {};
    uint16_t* H[4] = {};
    uint16_t* HT[4] = {};
    float* OUT = nullptr;
    float* Yb = nullptr;
    float* Gf[2] = {};
    uint16_t* Gb[2] = {};
    uint16_t* GT[2] = {};
    double* sse = nullptr;
    int sse_cap = 0;
    unsigned* status = nullptr;
    cudaStream_t st = nullptr;
    std::vector<void*> mem;

    template <typename T>
    T* alloc(size_t n) {
        void* p = nullptr;
        if (cudaMalloc(&p, sizeof(T) * (n ? n : 1)) != cudaSuccess) return nullptr;
        mem.push_back(p);
        return static_cast<T*>(p);
    }
    void release(void* p) {
        for (auto& q : mem)
            if (q == p) {
                cudaFree(q);
                q = nullptr;
            }
    }
    ~Trainer() {
        if (st) cudaStreamSynchronize(st);
        for (void* p : mem)
            if (p) cudaFree(p);
        if (st) cudaStreamDestroy(st);
    }
};

// one product; `splits` CTAs share K (the weight gradients only: their
// epilogue adds partial tiles)
static void gemm(Trainer* T, const GemmArgs& g, int splits = 1) {
    const int nt = g.N < kNt ? g.N : kNt;
    dim3 grid((unsigned)(g.M / kTile), (unsigned)(g.N / nt), (unsigned)splits);
    tr_gemm<<<grid, 128, kGemmSmem, T->st>>>(g);
    count_launch();
}

static GemmArgs gemm_args(Trainer* T, const uint16_t* A, int lda, const uint16_t* B, int ldb, int M, int N, int K,
                          int epi) {
    GemmArgs g{};
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.epi = epi;
    g.status = T->status;
    return g;
}

// forward (and the loss) of the batch rows idx[0..B) (device indices);
// with backward, the gradients into Gr; with update, an Adam step
static void run_batch(Trainer* T, const int* idx, int B, int sse_slot, bool backward, bool update) {
    const int Bp = (B + kTile - 1) / kTile * kTile;
    {
        const int n = Bp * kW;
        tr_gather<<<(n + 255) / 256, 256, 0, T->st>>>(T->X, T->Y, idx, B, Bp, T->H[0], T->HT[0], T->Yb);
        count_launch();
    }
    for (int l = 0; l < 3; ++l) {
        GemmArgs g = gemm_args(T, T->H[l], kW, T->Wb[l], kW, Bp, kW, kW, EPI_HIDDEN);
        g.bias = T->P + b_off(l);
        g.outb = T->H[l + 1];
        g.ldob = kW;
        g.outt = T->HT[l + 1];
        g.ldot = Bp;
        gemm(T, g);
    }
    {
        GemmArgs g = gemm_args(T, T->H[3], kW, T->Wb[3], kW, Bp, kOut, kW, EPI_OUT);
        g.bias = T->P + b_off(3);
        g.out = T->OUT;
        g.ldo = kOut;
        gemm(T, g);
    }
    {
        const int n = Bp * kOut;
        const float scale = (float)(2.0 / ((double)B * (double)T->n_out));
        tr_loss<<<(n + 255) / 256, 256, 0, T->st>>>(T->OUT, T->Yb, B, Bp, T->n_out, scale, T->Gf[0], T->Gb[0],
                                                     T->GT[0], T->sse + sse_slot);
        count_launch();
    }
    if (!backward) return;
    // the weight gradients accumulate partial tiles of their K splits
    cudaMemsetAsync(T->Gr, 0, sizeof(float) * kNW, T->st);
    const int splits = Bp >= 256 ? Bp / 256 : 1;     // about 256 batch rows (four slabs) per CTA
    int cur = 0;
    for (int l = 3; l >= 0; --l) {
        const int nl = rows_of(l);
        {
            GemmArgs g = gemm_args(T, T->HT[l], Bp, T->GT[cur], Bp, kW, nl, Bp, EPI_DW);
            g.out = T->Gr + w_off(l);
            g.ldo = kW;
            gemm(T, g, splits);
        }
        tr_bias_grad<<<nl, 256, 0, T->st>>>(T->Gf[cur], Bp, nl, T->Gr + b_off(l));
        count_launch();
        if (l > 0) {
            const int nx = cur ^ 1;
            GemmArgs g = gemm_args(T, T->Gb[cur], nl, T->WT[l], nl, Bp, kW, nl, EPI_DX);
            g.mask = T->H[l];
            g.ldm = kW;
            g.out = T->Gf[nx];
            g.ldo = kW;
            g.outb = T->Gb[nx];
            g.ldob = kW;
            g.outt = T->GT[nx];
            g.ldot = Bp;
            gemm(T, g);
            cur = nx;
        }
    }
    if (!update) return;
    T->step += 1;
    AdamArgs a;
    a.P = T->P;
    a.Gr = T->Gr;
    a.m = T->M;
    a.v = T->V;
    a.lr = (float)T->lr;
    a.b1 = (float)T->b1;
    a.b2 = (float)T->b2;
    a.eps = (float)T->eps;
    a.wd = (float)T->wd;
    a.c1 = (float)(1.0 / (1.0 - std::pow(T->b1, (double)T->step)));
    a.c2 = (float)(1.0 / (1.0 - std::pow(T->b2, (double)T->step)));
    for (int l = 0; l < 4; ++l) {
        a.Wb[l] = T->Wb[l];
        a.WT[l] = T->WT[l];
    }
    tr_adam<<<(kNP + 255) / 256, 256, 0, T->st>>>(a);
    count_launch();
}

static int finish(Trainer* T, const char* what) {
    cudaError_t e = cudaStreamSynchronize(T->st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return PP_E_CUDA;
    }
    unsigned s = 0;
    cudaMemcpy(&s, T->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (s & PP_ST_TIMEOUT) {
        set_error(std::string(what) + ": a bounded wait on the tensor cores expired");
        return PP_E_TIMEOUT;
    }
    return PP_OK;
}

// copies host indices to the device after checking them against the loaded rows
static int stage_indices(Trainer* T, const int32_t* idx, int n, const char* what) {
    if (!idx || n < 1) {
        set_error(std::string(what) + ": no rows");
        return PP_E_ARG;
    }
    if (T->rows < 1) {
        set_error(std::string(what) + ": no data loaded (pp_trainer_load)");
        return PP_E_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (idx[i] < 0 || idx[i] >= T->rows) {
            set_error(std::string(what) + ": row index out of range");
            return PP_E_ARG;
        }
    if (n > T->idx_cap) {
        if (T->idx) T->release(T->idx);
        T->idx = T->alloc<int>((size_t)n);
        T->idx_cap = T->idx ? n : 0;
        if (!T->idx) {
            set_error(std::string(what) + ": cudaMalloc failed");
            return PP_E_CUDA;
        }
    }
    const int nb = (n + T->batch - 1) / T->batch + 1;
    if (nb > T->sse_cap) {
        if (T->sse) T->release(T->sse);
        T->sse = T->alloc<double>((size_t)nb);
        T->sse_cap = T->sse ? nb : 0;
        if (!T->sse) {
            set_error(std::string(what) + ": cudaMalloc failed");
            return PP_E_CUDA;
        }
    }
    cudaMemcpyAsync(T->idx, idx, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, T->st);
    cudaMemsetAsync(T->sse, 0, sizeof(double) * (size_t)nb, T->st);
    cudaMemsetAsync(T->status, 0, sizeof(unsigned), T->st);
    return PP_OK;
}

static bool trainer_tc_attr() {
    static bool done = false;
    if (!done) done = cudaFuncSetAttribute(tr_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem) ==
                      cudaSuccess;
    return done;
}

}  // namespace pp

using namespace pp;

struct pp_trainer : public pp::Trainer {};

extern "C" {

int pp_trainer_create(const pp_train_opts* o, const float* const* w, const float* const* b, pp_trainer** out) {
    if (!o || !w || !b || !out || o->n_in < 1 || o->n_in > kW || o->n_out < 1 || o->n_out > kOut ||
        o->batch < 1 || o->batch > kMaxBatch || !(o->lr > 0) || !(o->beta1 >= 0 && o->beta1 < 1) ||
        !(o->beta2 >= 0 && o->beta2 < 1) || !(o->eps > 0) || !(o->weight_decay >= 0)) {
        set_error("bad argument to pp_trainer_create (n_in <= 256, n_out <= 32, batch <= 4096, lr > 0, "
                  "beta in [0, 1), eps > 0, weight_decay >= 0)");
        return PP_E_ARG;
    }
    for (int l = 0; l < 4; ++l)
        if (!w[l] || !b[l]) {
            set_error("pp_trainer_create: NULL weight or bias array");
            return PP_E_ARG;
        }
    *out = nullptr;
    pp_trainer* T = new pp_trainer();
    T->n_in = o->n_in;
    T->n_out = o->n_out;
    T->batch = o->batch;
    T->Bp = (o->batch + kTile - 1) / kTile * kTile;
    T->lr = o->lr;
    T->b1 = o->beta1;
    T->b2 = o->beta2;
    T->eps = o->eps;
    T->wd = o->weight_decay;
    bool ok = cudaStreamCreateWithFlags(&T->st, cudaStreamNonBlocking) == cudaSuccess && trainer_tc_attr();
    const size_t Bp = (size_t)T->Bp;
    if (ok) {
        T->P = T->alloc<float>(kNP);
        T->Gr = T->alloc<float>(kNP);
        T->M = T->alloc<float>(kNP);
        T->V = T->alloc<float>(kNP);
        for (int l = 0; l < 4; ++l) {
            T->Wb[l] = T->alloc<uint16_t>((size_t)rows_of(l) * kW);
            T->WT[l] = T->alloc<uint16_t>((size_t)rows_of(l) * kW);
            T->H[l] = T->alloc<uint16_t>(Bp * kW);
            T->HT[l] = T->alloc<uint16_t>(Bp * kW);
        }
        T->OUT = T->alloc<float>(Bp * kOut);
        T->Yb = T->alloc<float>(Bp * kOut);
        for (int i = 0; i < 2; ++i) {
            T->Gf[i] = T->alloc<float>(Bp * kW);
            T->Gb[i] = T->alloc<uint16_t>(Bp * kW);
            T->GT[i] = T->alloc<uint16_t>(Bp * kW);
        }
        T->status = T->alloc<unsigned>(1);
        ok = T->P && T->Gr && T->M && T->V && T->Wb[3] && T->WT[3] && T->H[3] && T->HT[3] && T->OUT && T->Yb &&
             T->Gf[1] && T->Gb[1] && T->GT[1] && T->status;
        for (int l = 0; l < 4 && ok; ++l) ok = T->Wb[l] && T->WT[l] && T->H[l] && T->HT[l];
    }
    if (!ok) {
        set_error("pp_trainer_create: CUDA allocation or stream creation failed");
        delete T;
        return PP_E_CUDA;
    }
    for (int l = 0; l < 4; ++l) {
        cudaMemcpyAsync(T->P + w_off(l), w[l], sizeof(float) * rows_of(l) * kW, cudaMemcpyHostToDevice, T->st);
        cudaMemcpyAsync(T->P + b_off(l), b[l], sizeof(float) * rows_of(l), cudaMemcpyHostToDevice, T->st);
    }
    cudaMemsetAsync(T->M, 0, sizeof(float) * kNP, T->st);
    cudaMemsetAsync(T->V, 0, sizeof(float) * kNP, T->st);
    cudaMemsetAsync(T->status, 0, sizeof(unsigned), T->st);
    AdamArgs a{};
    for (int l = 0; l < 4; ++l) {
        a.Wb[l] = T->Wb[l];
        a.WT[l] = T->WT[l];
    }
    tr_cast<<<(kNW + 255) / 256, 256, 0, T->st>>>(T->P, a);
    count_launch();
    int rc = finish(T, "pp_trainer_create");
    if (rc != PP_OK) {
        delete T;
        return rc;
    }
    *out = T;
    return PP_OK;
}

int pp_trainer_load(pp_trainer* T, const float* x, const float* y, int rows) {
    if (!T || !x || !y || rows < 1) {
        set_error("bad argument to pp_trainer_load");
        return PP_E_ARG;
    }
    if (T->X) T->release(T->X);
    if (T->Y) T->release(T->Y);
    T->rows = 0;
    T->X = T->alloc<uint16_t>((size_t)rows * kW);
    T->Y = T->alloc<float>((size_t)rows * kOut);
    float* xin = T->alloc<float>((size_t)rows * T->n_in);
    float* yin = T->alloc<float>((size_t)rows * T->n_out);
    if (!T->X || !T->Y || !xin || !yin) {
        set_error("pp_trainer_load: cudaMalloc failed");
        if (xin) T->release(xin);
        if (yin) T->release(yin);
        return PP_E_CUDA;
    }
    cudaMemcpyAsync(xin, x, sizeof(float) * (size_t)rows * T->n_in, cudaMemcpyHostToDevice, T->st);
    cudaMemcpyAsync(yin, y, sizeof(float) * (size_t)rows * T->n_out, cudaMemcpyHostToDevice, T->st);
    const size_t n = (size_t)rows * kW;
    tr_load<<<(unsigned)((n + 255) / 256), 256, 0, T->st>>>(xin, yin, rows, T->n_in, T->n_out, T->X, T->Y);
    count_launch();
    int rc = finish(T, "pp_trainer_load");
    T->release(xin);
    T->release(yin);
    if (rc == PP_OK) T->rows = rows;
    return rc;
}

int pp_trainer_gradients(pp_trainer* T, const int32_t* idx, int n, float* const* gw, float* const* gb,
                         double* loss) {
    if (!T || !gw || !gb || !loss || n > T->batch) {
        set_error("bad argument to pp_trainer_gradients (n <= the trainer's batch)");
        return PP_E_ARG;
    }
    for (int l = 0; l < 4; ++l)
        if (!gw[l] || !gb[l]) {
            set_error("pp_trainer_gradients: NULL output array");
            return PP_E_ARG;
        }
    int rc = stage_indices(T, idx, n, "pp_trainer_gradients");
    if (rc != PP_OK) return rc;
    run_batch(T, T->idx, n, 0, true, false);
    rc = finish(T, "pp_trainer_gradients");
    if (rc != PP_OK) return rc;
    for (int l = 0; l < 4; ++l) {
        cudaMemcpy(gw[l], T->Gr + w_off(l), sizeof(float) * rows_of(l) * kW, cudaMemcpyDeviceToHost);
        cudaMemcpy(gb[l], T->Gr + b_off(l), sizeof(float) * rows_of(l), cudaMemcpyDeviceToHost);
    }
    double s = 0;
    cudaMemcpy(&s, T->sse, sizeof(double), cudaMemcpyDeviceToHost);
    *loss = s / ((double)n * (double)T->n_out);
    return PP_OK;
}

int pp_trainer_epoch(pp_trainer* T, const int32_t* order, int n, double* mean_loss) {
    if (!T || !mean_loss) {
        set_error("bad argument to pp_trainer_epoch");
        return PP_E_ARG;
    }
    int rc = stage_indices(T, order, n, "pp_trainer_epoch");
    if (rc != PP_OK) return rc;
    int slot = 0;
    for (int s0 = 0; s0 < n; s0 += T->batch, ++slot) run_batch(T, T->idx + s0, std::min(T->batch, n - s0), slot, true, true);
    rc = finish(T, "pp_trainer_epoch");
    if (rc != PP_OK) return rc;
    std::vector<double> s((size_t)slot);
    cudaMemcpy(s.data(), T->sse, sizeof(double) * (size_t)slot, cudaMemcpyDeviceToHost);
    double tot = 0;
    for (double v : s) tot += v;
    *mean_loss = tot / ((double)n * (double)T->n_out);
    return PP_OK;
}

int pp_trainer_evaluate(pp_trainer* T, const int32_t* idx, int n, double* mse) {
    if (!T || !mse) {
        set_error("bad argument to pp_trainer_evaluate");
        return PP_E_ARG;
    }
    int rc = stage_indices(T, idx, n, "pp_trainer_evaluate");
    if (rc != PP_OK) return rc;
    int slot = 0;
    for (int s0 = 0; s0 < n; s0 += T->batch, ++slot) run_batch(T, T->idx + s0, std::min(T->batch, n - s0), slot, false, false);
    rc = finish(T, "pp_trainer_evaluate");
    if (rc != PP_OK) return rc;
    std::vector<double> s((size_t)slot);
    cudaMemcpy(s.data(), T->sse, sizeof(double) * (size_t)slot, cudaMemcpyDeviceToHost);
    double tot = 0;
    for (double v : s) tot += v;
    *mse = tot / ((double)n * (double)T->n_out);
    return PP_OK;
}

int pp_trainer_params(pp_trainer* T, float* const* w, uint16_t* const* wbits, float* const* b) {
    if (!T) {
        set_error("bad argument to pp_trainer_params");
        return PP_E_ARG;
    }
    cudaError_t e = cudaStreamSynchronize(T->st);
    if (e != cudaSuccess) {
        set_error(std::string("pp_trainer_params: ") + cudaGetErrorString(e));
        return PP_E_CUDA;
    }
    for (int l = 0; l < 4; ++l) {
        if (w && w[l]) cudaMemcpy(w[l], T->P + w_off(l), sizeof(float) * rows_of(l) * kW, cudaMemcpyDeviceToHost);
        if (wbits && wbits[l])
            cudaMemcpy(wbits[l], T->Wb[l], sizeof(uint16_t) * rows_of(l) * kW, cudaMemcpyDeviceToHost);
        if (b && b[l]) cudaMemcpy(b[l], T->P + b_off(l), sizeof(float) * rows_of(l), cudaMemcpyDeviceToHost);
    }
    return PP_OK;
}

int64_t pp_trainer_steps(pp_trainer* T) { return T ? (int64_t)T->step : -1; }

int pp_trainer_destroy(pp_trainer* T) {
    if (!T) {
        set_error("pp_trainer_destroy: NULL trainer");
        return PP_E_ARG;
    }
    delete T;
    return PP_OK;
}

}  // extern "C"
