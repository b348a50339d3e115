// BF16 MLP of the learned circuit proposal on the 5th-generation tensor
// cores: three hidden layers of 256 with ReLU and one output layer of 32,
// BF16 weights and activations, FP32 accumulation in tensor memory.
//
// One CTA of 128 threads takes 128 feature rows.  The activations of the
// current layer sit in shared memory as the MMA's A operand (128 x 256, K-major,
// no swizzle, 8-row x 16-byte core matrices), the layer's weights [out][in]
// as the B operand (N x 256, same layout).  Thread 0 issues the 16 K-steps of
// tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = 256 or 32, K = 16 each)
// into a 256-column TMEM accumulator and commits them to an mbarrier; the four
// warps then read their 32 TMEM lanes (rows) with tcgen05.ld, add the bias,
// apply ReLU, round to BF16 and write the next layer's A operand in place.
#include "pp_internal.h"
#include "pp_tc.cuh"

#include <cuda_bf16.h>

#include <string>
#include <vector>

namespace pp {

namespace {

constexpr int kW = 256;           // hidden width (and padded input width)
constexpr int kOut = 32;          // padded output width
constexpr int kRows = 128;        // rows per CTA (MMA M)
constexpr uint32_t kTmemCols = 256;

struct MlpSmem {
    __nv_bfloat16 a[kRows * kW];      // 64 KB activations (A operand)
    __nv_bfloat16 b[kW * kW];         // 128 KB weights of one layer (B operand)
    float bias[kW];
    uint64_t bar;
    uint32_t tmem_base;
};

using tc::smem_addr;
using tc::sdesc;
using tc::idesc_bf16;
using tc::kmajor_off;
using tc::mbar_wait_bounded;

// load `rows_n` rows of BF16 weights [out][in] (in = 256) into the K-major B operand
__device__ void load_weights(MlpSmem& s, const uint16_t* w, int rows_n, const float* bias) {
    const int chunks = rows_n * (kW / 8);              // 16-byte pieces (8 consecutive k)
    for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
        int n = q / (kW / 8), k8 = (q % (kW / 8)) * 8;
        uint4 v = *reinterpret_cast<const uint4*>(w + (size_t)n * kW + k8);
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(s.b) + kmajor_off(n, k8, rows_n)) = v;
    }
    for (int q = threadIdx.x; q < rows_n; q += blockDim.x) s.bias[q] = bias[q];
}

}  // namespace

struct MlpDev {
    const uint16_t* w[4];     // BF16 bits, [out][in]: 256x256 x3, 32x256
    const float* b[4];        // 256 x3, 32
    const double* mu_in;
    const double* sig_in;
    const double* mu_out;
    const double* sig_out;
    int n_in, n_out;
};

// feats: rows x n_in (double, raw features); out: rows x n_out (double, loads)
__global__ void __launch_bounds__(128, 1) mlp_forward_kernel(MlpDev m, const double* __restrict__ feats, int rows,
                                                             double* __restrict__ out, unsigned* status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    MlpSmem& s = *reinterpret_cast<MlpSmem*>(smraw);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int row0 = blockIdx.x * kRows;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) tc::mbar_init1(&s.bar);
    // standardised, BF16-rounded inputs (zero-padded rows and columns)
    for (int q = t; q < kRows * kW; q += blockDim.x) {
        int r = q / kW, k = q % kW;
        float v = 0.f;
        if (row0 + r < rows && k < m.n_in) v = (float)((feats[(size_t)(row0 + r) * m.n_in + k] - m.mu_in[k]) / m.sig_in[k]);
        *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(s.a) + kmajor_off(r, k, kRows)) =
            __float2bfloat16_rn(v);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s.tmem_base;
    uint32_t parity = 0;

    for (int layer = 0; layer < 4; ++layer) {
        const int N = layer < 3 ? kW : kOut;
        load_weights(s, m.w[layer], N, m.b[layer]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ab = smem_addr(s.a), bb = smem_addr(s.b);
            const uint32_t step_a = kRows * 32, step_b = (uint32_t)N * 32;
            const uint32_t idesc = idesc_bf16(kRows, N);
#pragma unroll 1
            for (int ks = 0; ks < kW / 16; ++ks) {
                uint64_t da = sdesc(ab + (uint32_t)ks * step_a, 128, 256);
                uint64_t db = sdesc(bb + (uint32_t)ks * step_b, 128, 256);
                tc::mma_bf16(tmem, da, db, idesc, ks > 0 ? 1u : 0u);
            }
            tc::mma_commit(&s.bar);
        }
        __syncwarp();
        // every thread waits; the block then agrees on the outcome
        const bool done = __syncthreads_and(mbar_wait_bounded(&s.bar, parity) ? 1 : 0) != 0;
        if (!done) {
            if (t == 0 && status) atomicOr(status, (unsigned)PP_ST_TIMEOUT);
            // the MMAs may still be in flight: one more bounded wait before TMEM is freed
            mbar_wait_bounded(&s.bar, parity);
            __syncthreads();
            break;
        }
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w + 31
        const int r = warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
            if (layer < 3) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float y = __uint_as_float(v[j]) + s.bias[c0 + j];
                    y = y > 0.f ? y : 0.f;
                    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(s.a) + kmajor_off(r, c0 + j, kRows)) =
                        __float2bfloat16_rn(y);
                }
            } else if (row0 + r < rows) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    int o = c0 + j;
                    if (o < m.n_out) {
                        double y = (double)(__uint_as_float(v[j]) + s.bias[o]);
                        out[(size_t)(row0 + r) * m.n_out + o] = y * m.sig_out[o] + m.mu_out[o];
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

size_t mlp_smem_bytes() { return sizeof(MlpSmem) + 1024; }

void launch_mlp_forward(const MlpDev& m, const double* feats, int rows, double* out, unsigned* status,
                        cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem_bytes());
        attr = true;
    }
    int blocks = (rows + kRows - 1) / kRows;
    mlp_forward_kernel<<<blocks, 128, mlp_smem_bytes(), st>>>(m, feats, rows, out, status);
    count_launch();
}

}  // namespace pp

// ---------------------------------------------------------------- period summaries
namespace pp {

constexpr int kBins = 32;

// electrons: per radial and axial bin the count and the sum of |v|^2
// (acc[0..31] radial v2 sums, acc[32..63] axial v2 sums; cnt[0..31] radial,
// cnt[32..63] axial)
__global__ void ml_bin_particles(ParticleBuf Pf, PBuf<double> Pd, int fp64, const int* nslot, int nr, double drm,
                                 double dzm, double r_max, double z_p, double* acc, unsigned long long* cnt) {
    __shared__ double s_v2[2 * kBins];
    __shared__ unsigned long long s_n[2 * kBins];
    for (int q = threadIdx.x; q < 2 * kBins; q += blockDim.x) {
        s_v2[q] = 0;
        s_n[q] = 0;
    }
    __syncthreads();
    const int n = nslot[0];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        uint32_t cell = fp64 ? Pd.cell[idx] : Pf.cell[idx];
        if (cell == kDead) continue;
        int iz = (int)(cell / (uint32_t)nr), ir = (int)(cell - (uint32_t)iz * (uint32_t)nr);
        double dr, dz, vr, vt, vz;
        if (fp64) {
            dr = Pd.dr[idx];
            dz = Pd.dz[idx];
            vr = Pd.vr[idx];
            vt = Pd.vt[idx];
            vz = Pd.vz[idx];
        } else {
            dr = Pf.dr[idx];
            dz = Pf.dz[idx];
            vr = Pf.vr[idx];
            vt = Pf.vt[idx];
            vz = Pf.vz[idx];
        }
        double r = ((double)ir + dr) * drm;
        double z = ((double)iz + dz) * dzm;
        double v2 = vr * vr + vt * vt + vz * vz;
        int br = min((int)((double)kBins * r / r_max), kBins - 1);
        int bz = min((int)((double)kBins * z / z_p), kBins - 1);
        atomicAdd(&s_v2[br], v2);
        atomicAdd(&s_v2[kBins + bz], v2);
        atomicAdd(&s_n[br], 1ull);
        atomicAdd(&s_n[kBins + bz], 1ull);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * kBins; q += blockDim.x) {
        if (s_n[q]) {
            atomicAdd(&acc[q], s_v2[q]);
            atomicAdd(&cnt[q], s_n[q]);
        }
    }
}

// current amplitude on the plasma nodes (acc[64..95] radial numerators,
// acc[96..127] axial numerators, acc[128..159] radial volumes, acc[160..191] axial)
__global__ void ml_bin_nodes(const double* Jc, const double* Js, const double* vol, int NR, int i_win, double drm,
                             double dzm, double r_max, double z_p, double* acc) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (i_win + 1) * NR) return;
    int i = n / NR, j = n % NR;
    double rn = j * drm, zn = i * dzm;
    if (rn >= r_max || zn >= z_p) return;
    double J = sqrt(Jc[n] * Jc[n] + Js[n] * Js[n]);
    int br = min((int)((double)kBins * rn / r_max), kBins - 1);
    int bz = min((int)((double)kBins * zn / z_p), kBins - 1);
    atomicAdd(&acc[2 * kBins + br], J * vol[n]);
    atomicAdd(&acc[3 * kBins + bz], J * vol[n]);
    atomicAdd(&acc[4 * kBins + br], vol[n]);
    atomicAdd(&acc[5 * kBins + bz], vol[n]);
}

// feature vector (the order of pp_ml_configure's description)
__global__ void ml_make_features(const DevState* st, const double* acc, const unsigned long long* cnt, int N,
                                 double weight, double r_max, double z_p, double* feat) {
    const int t = threadIdx.x;
    const int nx = 2 * (2 * N + 1);
    const double pi = 3.14159265358979323846;
    if (t < nx) feat[t] = st->x[t];
    if (t < kBins) {
        int b = t;
        double e0 = r_max * b / kBins, e1 = r_max * (b + 1) / kBins;
        double vol_r = pi * (e1 * e1 - e0 * e0) * z_p;
        double vol_z = pi * (r_max * r_max) * z_p / kBins;
        double nr_ = (double)cnt[b], nz_ = (double)cnt[kBins + b];
        double ne_r = nr_ * weight / vol_r, ne_z = nz_ * weight / vol_z;
        const double te_scale = 9.1093837015e-31 / (3.0 * 1.602176634e-19);
        feat[nx + b] = log10(fmax(ne_r, 1e10));
        feat[nx + kBins + b] = log10(fmax(ne_z, 1e10));
        feat[nx + 2 * kBins + b] = nr_ > 0 ? te_scale * acc[b] / nr_ : 0.0;
        feat[nx + 3 * kBins + b] = nz_ > 0 ? te_scale * acc[kBins + b] / nz_ : 0.0;
        double dr_ = acc[4 * kBins + b], dz_ = acc[5 * kBins + b];
        feat[nx + 4 * kBins + b] = dr_ > 0 ? acc[2 * kBins + b] / dr_ : 0.0;
        feat[nx + 5 * kBins + b] = dz_ > 0 ? acc[3 * kBins + b] / dz_ : 0.0;
    }
}

void ml_features(Cell* c, cudaStream_t st) {
    const double z_p = c->i_win * c->dz;
    cudaMemsetAsync(c->d_ml_acc, 0, sizeof(double) * 8 * kBins, st);
    cudaMemsetAsync(c->d_ml_cnt, 0, sizeof(unsigned long long) * 2 * kBins, st);
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    ml_bin_particles<<<nsm * 4, 256, 0, st>>>(c->pb[0][c->cur[0]], c->pd[0][c->cur[0]], c->fp64 ? 1 : 0, c->d_nslot,
                                               c->nr, c->dr, c->dz, c->cfg.r_max, z_p, c->d_ml_acc, c->d_ml_cnt);
    int nn = (c->i_win + 1) * c->NR;
    ml_bin_nodes<<<(nn + 255) / 256, 256, 0, st>>>(c->d_Jc, c->d_Js, c->d_vol, c->NR, c->i_win, c->dr, c->dz,
                                                   c->cfg.r_max, z_p, c->d_ml_acc);
    ml_make_features<<<1, 64, 0, st>>>(c->d_st, c->d_ml_acc, c->d_ml_cnt, c->nturns, c->cfg.weight[0],
                                       c->cfg.r_max, z_p, c->d_ml_feat);
    count_launch(3);
    c->ml_have_features = true;
}

static MlpDev cell_mlp(const Cell* c) {
    MlpDev m;
    for (int l = 0; l < 4; ++l) {
        m.w[l] = c->d_ml_w[l];
        m.b[l] = c->d_ml_b[l];
    }
    m.mu_in = c->d_ml_norm;
    m.sig_in = c->d_ml_norm + 256;
    m.mu_out = c->d_ml_norm + 512;
    m.sig_out = c->d_ml_norm + 544;
    m.n_in = c->ml_n_in;
    m.n_out = c->ml_n_out;
    return m;
}

void ml_predict(Cell* c, cudaStream_t st) {
    launch_mlp_forward(cell_mlp(c), c->d_ml_feat, 1, c->d_ml_pred, &c->d_st->status, st);
}

static int check_mlp(const pp_mlp* m) {
    if (!m || m->n_in < 1 || m->n_in > kW || m->n_out < 1 || m->n_out > kOut) return 0;
    for (int l = 0; l < 4; ++l)
        if (!m->w[l] || !m->b[l]) return 0;
    return m->mu_in && m->sig_in && m->mu_out && m->sig_out;
}

int ml_configure(Cell* c, const pp_mlp* m, double alpha_ml, int collect) {
    cudaDeviceSynchronize();
    const int nfeat = 2 * (2 * c->nturns + 1) + 6 * kBins;
    if (m && (!check_mlp(m) || m->n_in != nfeat || m->n_out != 4 * c->nturns)) {
        set_error("MLP sizes do not match this cell (n_in = 2(2N+1) + 192, n_out = 4N)");
        return PP_E_ARG;
    }
    if (!c->d_ml_feat) {
        c->d_ml_feat = c->alloc<double>(kW);
        c->d_ml_pred = c->alloc<double>(kOut);
        c->d_ml_acc = c->alloc<double>(8 * kBins);
        c->d_ml_cnt = c->alloc<unsigned long long>(2 * kBins);
        c->d_ml_norm = c->alloc<double>(2 * kW + 2 * kOut);
        for (int l = 0; l < 4; ++l) {
            int rows = l < 3 ? kW : kOut;
            c->d_ml_w[l] = c->alloc<uint16_t>((size_t)rows * kW);
            c->d_ml_b[l] = c->alloc<float>(rows);
        }
        if (!c->d_ml_b[3]) {
            set_error("cudaMalloc failed for the MLP");
            return PP_E_CUDA;
        }
    }
    c->ml_collect = collect != 0 || m != nullptr;
    c->ml_model = m != nullptr;
    c->alpha_ml = alpha_ml;
    c->ml_n_in = nfeat;
    c->ml_n_out = 4 * c->nturns;
    if (m) {
        for (int l = 0; l < 4; ++l) {
            int rows = l < 3 ? kW : kOut;
            cudaMemcpy(c->d_ml_w[l], m->w[l], sizeof(uint16_t) * rows * kW, cudaMemcpyHostToDevice);
            cudaMemcpy(c->d_ml_b[l], m->b[l], sizeof(float) * rows, cudaMemcpyHostToDevice);
        }
        cudaMemcpy(c->d_ml_norm, m->mu_in, sizeof(double) * m->n_in, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_ml_norm + 256, m->sig_in, sizeof(double) * m->n_in, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_ml_norm + 512, m->mu_out, sizeof(double) * m->n_out, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_ml_norm + 544, m->sig_out, sizeof(double) * m->n_out, cudaMemcpyHostToDevice);
    }
    // a new model starts its gate afresh
    int zero[4] = {0, 0, 0, 0};
    cudaMemcpy(&c->d_st->ml_has_pred, zero, sizeof(zero), cudaMemcpyHostToDevice);
    c->graph_cur[0] = c->graph_cur[1] = -1;     // the period graph changes
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        set_error(std::string("pp_ml_configure: ") + cudaGetErrorString(e));
        return PP_E_CUDA;
    }
    return PP_OK;
}

}  // namespace pp

using namespace pp;

extern "C" {

int pp_mlp_forward(const pp_mlp* m, const double* feats, int rows, double* out) {
    if (!check_mlp(m) || !feats || !out || rows < 1) {
        set_error("bad argument to pp_mlp_forward");
        return PP_E_ARG;
    }
    std::vector<void*> mem;
    auto dalloc = [&](size_t bytes) {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return (void*)nullptr;
        mem.push_back(p);
        return p;
    };
    MlpDev d;
    bool ok = true;
    for (int l = 0; l < 4; ++l) {
        int r = l < 3 ? kW : kOut;
        uint16_t* w = (uint16_t*)dalloc(sizeof(uint16_t) * r * kW);
        float* b = (float*)dalloc(sizeof(float) * r);
        ok = ok && w && b;
        if (!ok) break;
        cudaMemcpy(w, m->w[l], sizeof(uint16_t) * r * kW, cudaMemcpyHostToDevice);
        cudaMemcpy(b, m->b[l], sizeof(float) * r, cudaMemcpyHostToDevice);
        d.w[l] = w;
        d.b[l] = b;
    }
    double* norm = ok ? (double*)dalloc(sizeof(double) * (2 * m->n_in + 2 * m->n_out)) : nullptr;
    double* df = ok ? (double*)dalloc(sizeof(double) * (size_t)rows * m->n_in) : nullptr;
    double* dout = ok ? (double*)dalloc(sizeof(double) * (size_t)rows * m->n_out) : nullptr;
    unsigned* dst = ok ? (unsigned*)dalloc(sizeof(unsigned)) : nullptr;
    int rc = PP_OK;
    if (!norm || !df || !dout || !dst) {
        set_error("cudaMalloc failed in pp_mlp_forward");
        rc = PP_E_CUDA;
    } else {
        cudaMemcpy(norm, m->mu_in, sizeof(double) * m->n_in, cudaMemcpyHostToDevice);
        cudaMemcpy(norm + m->n_in, m->sig_in, sizeof(double) * m->n_in, cudaMemcpyHostToDevice);
        cudaMemcpy(norm + 2 * m->n_in, m->mu_out, sizeof(double) * m->n_out, cudaMemcpyHostToDevice);
        cudaMemcpy(norm + 2 * m->n_in + m->n_out, m->sig_out, sizeof(double) * m->n_out, cudaMemcpyHostToDevice);
        cudaMemcpy(df, feats, sizeof(double) * (size_t)rows * m->n_in, cudaMemcpyHostToDevice);
        cudaMemset(dst, 0, sizeof(unsigned));
        d.mu_in = norm;
        d.sig_in = norm + m->n_in;
        d.mu_out = norm + 2 * m->n_in;
        d.sig_out = norm + 2 * m->n_in + m->n_out;
        d.n_in = m->n_in;
        d.n_out = m->n_out;
        launch_mlp_forward(d, df, rows, dout, dst, 0);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            set_error(std::string("pp_mlp_forward: ") + cudaGetErrorString(e));
            rc = PP_E_CUDA;
        } else {
            unsigned s = 0;
            cudaMemcpy(&s, dst, sizeof(unsigned), cudaMemcpyDeviceToHost);
            cudaMemcpy(out, dout, sizeof(double) * (size_t)rows * m->n_out, cudaMemcpyDeviceToHost);
            if (s & PP_ST_TIMEOUT) {
                set_error("a bounded wait on the tensor cores expired");
                rc = PP_E_TIMEOUT;
            }
        }
    }
    for (void* p : mem) cudaFree(p);
    return rc;
}

int pp_ml_configure(pp_cell* h, const pp_mlp* m, double alpha_ml, int collect) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !(alpha_ml > 0.0 && alpha_ml <= 1.0)) {
        set_error("bad argument to pp_ml_configure (alpha_ml in (0, 1])");
        return PP_E_ARG;
    }
    if (c->nharm > 1) {
        set_error("pp_ml_configure: the proposal predicts the fundamental's loads; the cell retains harmonics");
        return PP_E_CONFIG;
    }
    if (c->weighted) {
        set_error("pp_ml_configure: the summaries count unweighted macroparticles; the cell has per-particle weights");
        return PP_E_CONFIG;
    }
    return ml_configure(c, m, alpha_ml, collect);
}

int pp_get_ml_features(pp_cell* h, double* out, int cap, int* n, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !out || !n || !c->ml_have_features) {
        set_error("no features: enable collection with pp_ml_configure or call pp_ml_features_now");
        return PP_E_ARG;
    }
    *n = c->ml_n_in;
    if (cap < c->ml_n_in) {
        set_error("output array too small");
        return PP_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemcpyAsync(out, c->d_ml_feat, sizeof(double) * c->ml_n_in, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error(std::string("pp_get_ml_features: ") + cudaGetErrorString(e));
        return PP_E_CUDA;
    }
    return PP_OK;
}

int pp_ml_features_now(pp_cell* h, void* stream) {
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !c->d_ml_feat) {
        set_error("call pp_ml_configure first");
        return PP_E_ARG;
    }
    ml_features(c, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("pp_ml_features_now: ") + cudaGetErrorString(e));
        return PP_E_CUDA;
    }
    return PP_OK;
}

}  // extern "C"
