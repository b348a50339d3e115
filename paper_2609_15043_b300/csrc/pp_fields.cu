// Field kernels: separable direct solver (radial generalised eigenbasis x
// tridiagonal in z), the Poisson FP64 residual refinement with a capacitance
// correction for the equipotential turn nodes, the Helmholtz FP64 solve, node
// fields for the gather, turn charges and the per-step harmonic accumulation.
#include "pp_internal.h"

#include <atomic>

#include <cmath>
#include <string>

namespace pp {

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* a, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double kahan_add(double& sum, double& comp, double v) {
    double y = v - comp;
    double t = sum + y;
    comp = (t - sum) - y;
    sum = t;
    return t;
}

// ---------------------------------------------------------------- GEMM
// C[rows x N] = A[rows x K] * B[K x N], row-major, 32x32 tiles.
template <typename T>
__global__ void gemm_rm(const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ C,
                        int rows, int K, int N, const int* skip) {
    if (skip && *skip) return;
    __shared__ T As[32][33];
    __shared__ T Bs[32][33];
    int tx = threadIdx.x, ty = threadIdx.y;          // 32 x 8
    int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    T acc[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int q = 0; q < 4; ++q) {
            int r = ty + 8 * q;
            As[r][tx] = (r0 + r < rows && k0 + tx < K) ? A[(size_t)(r0 + r) * K + k0 + tx] : T(0);
            Bs[r][tx] = (k0 + r < K && c0 + tx < N) ? B[(size_t)(k0 + r) * N + c0 + tx] : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            T b = Bs[k][tx];
            for (int q = 0; q < 4; ++q) acc[q] += As[ty + 8 * q][k] * b;
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q) {
        int r = r0 + ty + 8 * q, cc = c0 + tx;
        if (r < rows && cc < N) C[(size_t)r * N + cc] = acc[q];
    }
}

// The two products of a Poisson sweep, C = A B with 32 x 32 output tiles:
// K is taken in slabs of 128 whose 32 loads per thread are all issued before
// any of them is stored to shared memory, so a slab costs one memory latency.
// With `check` the block first takes the sweep's convergence decision from
// the residual norms (identical in every block; all return when converged).
template <bool check>
__global__ void __launch_bounds__(256) gemm_sweep(const float* __restrict__ A, const float* __restrict__ B,
                                                  float* __restrict__ C, int rows, int K, int N, DevState* st,
                                                  int sweep, double tol, int* done) {
    if (*done) return;
    if (check) {
        double rn = __longlong_as_double((long long)st->pnorm[2 * sweep]);
        double sn = __longlong_as_double((long long)st->pnorm[2 * sweep + 1]);
        double rel = (sn > 0) ? rn / sn : 0.0;
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
            st->prel = rel;
            st->piters = sweep;
            if (rel <= tol) *done = 1;
        }
        if (rel <= tol) return;
    }
    constexpr int KS = 128;
    __shared__ float As[32][KS + 1];
    __shared__ float Bs[KS][33];
    const int tx = threadIdx.x, ty = threadIdx.y;          // 32 x 8
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += KS) {
        float ra[4][4], rb[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = ty + 8 * q, k = k0 + 32 * j + tx, kr = k0 + 32 * j + r;
                ra[j][q] = (r0 + r < rows && k < K) ? A[(size_t)(r0 + r) * K + k] : 0.f;
                rb[j][q] = (kr < K && c0 + tx < N) ? B[(size_t)kr * N + c0 + tx] : 0.f;
            }
        if (k0) __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                As[ty + 8 * q][32 * j + tx] = ra[j][q];
                Bs[32 * j + ty + 8 * q][tx] = rb[j][q];
            }
        __syncthreads();
        const int kn = min(KS, K - k0);
#pragma unroll 8
        for (int k = 0; k < kn; ++k) {
            float b = Bs[k][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += As[ty + 8 * q][k] * b;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int r = r0 + ty + 8 * q, cc = c0 + tx;
        if (r < rows && cc < N) C[(size_t)r * N + cc] = acc[q];
    }
}

// Thomas sweep per mode with precomputed factors.  A block takes MB modes:
// all of their rows of f, c' and 1/denominator are staged in shared memory
// with coalesced row loads, one warp runs the two dependent recurrences out of
// shared memory (one lane per mode), and the result is written back row-wise.
template <typename T>
__global__ void tri_solve(const T* __restrict__ f, T* __restrict__ x, const T* __restrict__ cp,
                          const T* __restrict__ invd, const T* __restrict__ lo, int rows, int M, int MB,
                          const int* skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    T* sf = reinterpret_cast<T*>(smem_raw);          // rows x MB
    T* sc = sf + (size_t)rows * MB;
    T* sd = sc + (size_t)rows * MB;
    T* sl = sd + (size_t)rows * MB;                  // rows
    const int m0 = blockIdx.x * MB;
    const int nm = min(MB, M - m0);
    for (int q = threadIdx.x; q < rows * MB; q += blockDim.x) {
        int i = q / MB, mm = q % MB;
        if (mm < nm) {
            size_t k = (size_t)i * M + m0 + mm;
            sf[q] = f[k];
            sc[q] = cp[k];
            sd[q] = invd[k];
        }
    }
    for (int i = threadIdx.x; i < rows; i += blockDim.x) sl[i] = lo[i];
    __syncthreads();
    if (threadIdx.x < nm) {
        const int mm = threadIdx.x;
        T y = 0;
        for (int i = 0; i < rows; ++i) {
            y = (sf[i * MB + mm] - sl[i] * y) * sd[i * MB + mm];
            sf[i * MB + mm] = y;
        }
        T xn = sf[(rows - 1) * MB + mm];
        for (int i = rows - 2; i >= 0; --i) {
            xn = sf[i * MB + mm] - sc[i * MB + mm] * xn;
            sf[i * MB + mm] = xn;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < rows * MB; q += blockDim.x) {
        int i = q / MB, mm = q % MB;
        if (mm < nm) x[(size_t)i * M + m0 + mm] = sf[q];
    }
}

template <typename T>
static int tri_modes_per_block(int rows) {
    // 3 row arrays per mode in at most ~200 KB of shared memory
    int mb = 32;
    while (mb > 1 && (size_t)(3 * mb + 1) * rows * sizeof(T) > 200 * 1024) mb >>= 1;
    return mb;
}

// Parallel cyclic reduction of the per-mode z systems with precomputed level
// coefficients (mode-major: al[(m L + l) rows + i]).  One block per mode; a
// thread owns rows i = t + k*blockDim for k < EPT and holds every level's
// coefficients in registers, so a level is two shared loads and two FMAs.
template <int EPT>
__global__ void __launch_bounds__(256) pcr_solve(const float* __restrict__ f, float* __restrict__ x,
                                                 const float* __restrict__ al, const float* __restrict__ ga,
                                                 const float* __restrict__ ib, int rows, int M, int L, const int* skip) {
    if (skip && *skip) return;
    __shared__ float d[2][256 * EPT];
    const int m = blockIdx.x;
    float ra[kMaxPcrLevels][EPT], rg[kMaxPcrLevels][EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        int i = threadIdx.x + k * 256;
        bool ok = i < rows;
        d[0][threadIdx.x + k * 256] = ok ? f[(size_t)i * M + m] : 0.f;
#pragma unroll
        for (int l = 0; l < kMaxPcrLevels; ++l) {
            bool lk = ok && l < L;
            ra[l][k] = lk ? al[((size_t)m * L + l) * rows + i] : 0.f;
            rg[l][k] = lk ? ga[((size_t)m * L + l) * rows + i] : 0.f;
        }
    }
    __syncthreads();
    int cur = 0;
#pragma unroll
    for (int l = 0; l < kMaxPcrLevels; ++l) {
        if (l >= L) break;
        const int st = 1 << l;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            int i = threadIdx.x + k * 256;
            if (i < rows) {
                float v = d[cur][i];
                if (i - st >= 0) v += ra[l][k] * d[cur][i - st];
                if (i + st < rows) v += rg[l][k] * d[cur][i + st];
                d[cur ^ 1][i] = v;
            }
        }
        __syncthreads();
        cur ^= 1;
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        int i = threadIdx.x + k * 256;
        if (i < rows) x[(size_t)i * M + m] = d[cur][i] * ib[(size_t)m * rows + i];
    }
}

static void launch_pcr(const Cell* c, const float* f, float* x, cudaStream_t st, const int* skip) {
    int rows = c->ps.rows, M = c->ps.M, L = c->pcr_levels;
    if (rows <= 256)
        pcr_solve<1><<<M, 256, 0, st>>>(f, x, c->d_pcr_a, c->d_pcr_g, c->d_pcr_ib, rows, M, L, skip);
    else if (rows <= 512)
        pcr_solve<2><<<M, 256, 0, st>>>(f, x, c->d_pcr_a, c->d_pcr_g, c->d_pcr_ib, rows, M, L, skip);
    else
        pcr_solve<4><<<M, 256, 0, st>>>(f, x, c->d_pcr_a, c->d_pcr_g, c->d_pcr_ib, rows, M, L, skip);
}

template <typename T>
void sep_solve(const SepSolver<T>& s, const T* rhs, T* out, cudaStream_t st, const int* skip) {
    dim3 blk(32, 8), grd((s.M + 31) / 32, (s.rows + 31) / 32);
    gemm_rm<T><<<grd, blk, 0, st>>>(rhs, s.Vf, s.t0, s.rows, s.M, s.M, skip);
    int mb = tri_modes_per_block<T>(s.rows);
    size_t shm = (size_t)(3 * mb + 1) * s.rows * sizeof(T);
    // the large shared-memory attribute, once per device (an attribute belongs
    // to the device that is current when it is set); concurrent first calls
    // set it twice, which is harmless
    static std::atomic<unsigned long long> attr_devs[2];
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(attr_devs[sizeof(T) == 8].load() & bit)) {
        cudaFuncSetAttribute(tri_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr_devs[sizeof(T) == 8].fetch_or(bit);
    }
    tri_solve<T><<<(s.M + mb - 1) / mb, 256, shm, st>>>(s.t0, s.t1, s.cp, s.invd, s.lo, s.rows, s.M, mb, skip);
    gemm_rm<T><<<grd, blk, 0, st>>>(s.t1, s.Vb, out, s.rows, s.M, s.M, skip);
    count_launch(3);
}
template void sep_solve<float>(const SepSolver<float>&, const float*, float*, cudaStream_t, const int*);
template void sep_solve<double>(const SepSolver<double>&, const double*, double*, cudaStream_t, const int*);

// ---------------------------------------------------------------- Poisson

__device__ __forceinline__ double turn_target(const DevState* st, const double* ext, int k, int nt,
                                              double cs, double sn) {
    if (ext) return ext[k];
    // Eq. dirichlet: phi_k = V_c cos + V_s sin with V = V_c - i V_s, plus the
    // retained harmonics
    double vr = st->x[2 * (1 + nt + k)], vi = st->x[2 * (1 + nt + k) + 1];
    const double v1 = vr * cs + (-vi) * sn;
    return st->nharm > 1 ? v1 + harm_turn_sum(st, k, nt, cs, sn) : v1;
}

struct PoisArgs {
    const double* phi;
    const float* rho;
    const float* rho_i;            // ion charge (added when set)
    const double* rho64;           // node charge of the plain FP64 form (used when set)
    const double* rho64_i;
    const double* win;
    const double* eps_row;
    const double* az;
    const double* arp;
    const double* arm;
    const signed char* turn_mask;   // per node: -1 or turn index
    float* r32;
    int NR, NZ, M;
    double inv2pieps0;
    unsigned long long* norm;      // [2]: max|r|, max term scale
    const int* done;
    const DevState* st;            // turn potentials from the applied circuit state
    const double* ext;             // or from an explicit array
    int nt;
    double cs, sn;
};

// r = b - A phi on the interior unknowns (i = 1..NZ-2, j = 0..NR-2).  Turn
// nodes contribute their Dirichlet mismatch (target - phi) times the diagonal
// coefficient to the norm and get r = 0 in the FP32 right-hand side (the
// capacitance step imposes their values).  The relative residual is
// max|r| / max(|b| + sum |A_ij phi_j|) (a componentwise scale).
__global__ void poisson_residual(PoisArgs a) {
    if (*a.done) return;
    int rows = a.NZ - 2;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    double rmax = 0, smax = 0;
    if (idx < rows * a.M) {
        int i = idx / a.M + 1, j = idx % a.M;
        int n = i * a.NR + j;
        double epz = a.eps_row[i], emz = a.eps_row[i - 1];
        double eb = 0.5 * (emz + epz);
        int k = a.turn_mask[n];
        if (k >= 0) {
            a.r32[idx] = 0.f;
            double diag = a.az[j] * (epz + emz) + eb * (a.arp[j] + a.arm[j]);
            double tgt = turn_target(a.st, a.ext, k, a.nt, a.cs, a.sn);
            rmax = fabs(tgt - a.phi[n]) * diag;
            smax = fabs(tgt) * diag;
        } else {
            double pc = a.phi[n];
            double t1 = a.az[j] * epz * (a.phi[n + a.NR] - pc);
            double t2 = a.az[j] * emz * (a.phi[n - a.NR] - pc);
            double t3 = eb * a.arp[j] * (a.phi[n + 1] - pc);
            double t4 = (j > 0) ? eb * a.arm[j] * (a.phi[n - 1] - pc) : 0.0;
            double q = a.rho64 ? a.rho64[n] + (a.rho64_i ? a.rho64_i[n] : 0.0)
                               : (double)a.rho[n] + (a.rho_i ? (double)a.rho_i[n] : 0.0);
            double b = -(q + a.win[n]) * a.inv2pieps0;
            double r = b - (((t1 + t2) + t3) + t4);
            a.r32[idx] = (float)r;
            rmax = fabs(r);
            smax = fabs(b) + fabs(t1) + fabs(t2) + fabs(t3) + fabs(t4);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(&a.norm[0], rmax);
        atomic_max_nonneg(&a.norm[1], smax);
    }
}

// decides convergence from the norms of this sweep (runs before the solve)
__global__ void poisson_check(DevState* st, int sweep, double tol, int* done, int final_sweep) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (*done) return;
    double r = __longlong_as_double((long long)st->pnorm[2 * sweep]);
    double s = __longlong_as_double((long long)st->pnorm[2 * sweep + 1]);
    double rel = (s > 0) ? r / s : 0.0;
    st->prel = rel;
    st->piters = sweep;
    if (rel <= tol) {
        *done = 1;
    } else if (final_sweep) {
        st->status |= PP_ST_NOCONV;
    }
}

// sigma = G^-1 (target - phi_T - d0_T)
__global__ void poisson_cap(const DevState* st, const double* ext, const double* phi, const float* d0,
                            const int* tn_node, const int* tn_int, const int* tn_k, const double* Ginv,
                            double* sigma, int K, int nt, double cs, double sn, const int* done) {
    if (*done) return;
    __shared__ double rT[kMaxCapNodes];
    int t = threadIdx.x;
    if (t < K) rT[t] = turn_target(st, ext, tn_k[t], nt, cs, sn) - phi[tn_node[t]] - (double)d0[tn_int[t]];
    __syncthreads();
    if (t < K) {
        double s = 0;
        for (int u = 0; u < K; ++u) s += Ginv[t * K + u] * rT[u];
        sigma[t] = s;
    }
}

// the turn nodes take their Dirichlet values before the sweeps, so every
// later correction there is zero and no kernel of the solve writes them
__global__ void poisson_set_turns(double* phi, const int* tn_node, const int* tn_k, int K, DevState* st,
                                  const double* ext, int nt, double cs, double sn) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    // fresh refinement bookkeeping for this solve
    if (t < 2 * 16) st->pnorm[t] = 0ull;
    if (t == 0) st->pdone = 0;
    if (t < K) phi[tn_node[t]] = turn_target(st, ext, tn_k[t], nt, cs, sn);
}

// phi += d0 + Z sigma as poisson_update_cap, with the K corrections of an
// unknown read as contiguous float4s (Zt: unknown-major, K padded to Kp)
__global__ void poisson_update_zt(double* phi, const float* d0, const float* __restrict__ Zt, const double* Ginv,
                                  const int* tn_int, int K, int Kp, int rows, int M, int NR,
                                  const signed char* turn_mask, const int* done) {
    if (*done) return;
    __shared__ double s_r[kMaxCapNodes];
    __shared__ double s_sig[kMaxCapNodes + 4];
    // the thread's own unknown is read first, so its latency overlaps sigma's
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = idx < rows * M;
    const int n = act ? (idx / M + 1) * NR + idx % M : 0;
    const bool free_node = act && turn_mask[n] < 0;
    double d = free_node ? (double)d0[idx] : 0.0;
    for (int q = threadIdx.x; q < K; q += blockDim.x) s_r[q] = -(double)d0[tn_int[q]];
    for (int q = K + threadIdx.x; q < Kp; q += blockDim.x) s_sig[q] = 0.0;
    __syncthreads();
    // sigma = G^-1 s_r: one warp per row, lanes across the row (independent loads)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = warp; q < K; q += nw) {
        double part = 0.0;
        for (int u = lane; u < K; u += 32) part += Ginv[q * K + u] * s_r[u];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) s_sig[q] = part;
    }
    __syncthreads();
    if (!free_node) return;
    // Z sigma in FP32: it corrects the FP32 inner solve, whose error the FP64
    // residual of the next sweep measures anyway (FP64 rate is low on B300)
    const float4* z = reinterpret_cast<const float4*>(Zt + (size_t)idx * Kp);
    float zc = 0.f;
#pragma unroll 4
    for (int t = 0; t < Kp / 4; ++t) {
        float4 v = z[t];
        zc += (float)s_sig[4 * t] * v.x + (float)s_sig[4 * t + 1] * v.y + (float)s_sig[4 * t + 2] * v.z +
              (float)s_sig[4 * t + 3] * v.w;
    }
    phi[n] += d + (double)zc;
}

// phi += d0 + Z sigma with sigma = G^-1 (-d0_T) computed by every block
// (the turn nodes already hold their targets)
__global__ void poisson_update_cap(double* phi, const float* d0, const float* Z, const double* Ginv,
                                   const int* tn_int, int K, int rows, int M, int NR,
                                   const signed char* turn_mask, const int* done) {
    if (*done) return;
    __shared__ double s_r[kMaxCapNodes];
    __shared__ double s_sig[kMaxCapNodes];
    for (int q = threadIdx.x; q < K; q += blockDim.x) s_r[q] = -(double)d0[tn_int[q]];
    __syncthreads();
    for (int q = threadIdx.x; q < K; q += blockDim.x) {
        double sg = 0;
        for (int u = 0; u < K; ++u) sg += Ginv[q * K + u] * s_r[u];
        s_sig[q] = sg;
    }
    __syncthreads();
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * M) return;
    int n = (idx / M + 1) * NR + idx % M;
    if (turn_mask[n] >= 0) return;
    double d = (double)d0[idx];
    size_t stride = (size_t)rows * M;
    for (int t = 0; t < K; ++t) d += s_sig[t] * (double)Z[t * stride + idx];
    phi[n] += d;
}

__global__ void poisson_update(double* phi, const float* d0, const float* Z, const double* sigma, int K,
                               int rows, int M, int NR, const signed char* turn_mask, const DevState* st,
                               const double* ext, int nt, double cs, double sn, const int* done) {
    if (*done) return;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * M) return;
    int i = idx / M + 1, j = idx % M;
    int n = i * NR + j;
    int k = turn_mask[n];
    if (k >= 0) {
        phi[n] = turn_target(st, ext, k, nt, cs, sn);
        return;
    }
    double d = (double)d0[idx];
    size_t stride = (size_t)rows * M;
    for (int t = 0; t < K; ++t) d += sigma[t] * (double)Z[t * stride + idx];
    phi[n] += d;
}

// ---------------------------------------------------------------- node fields
// what the step's field preparation imposes for the following Poisson solve
struct TurnSet {
    double* phi;
    const int* tn_node;
    const int* tn_k;
    int K, nt;
    DevState* st;
    double cs, sn;
};

// the retained harmonics' composed fields at the step's phase
struct HarmFields {
    const double* Ech;      // (nh) x 2 x nodes: E_c, E_ss
    const double* Bh;       // (nh) x 4 x nodes
    HarmPhase ph;           // cos m theta, sin m theta
};

// Per plasma cell 5 x 4 values (Er, Ez, Etheta, Br, Bz at corners 00, 01, 10,
// 11).  A block takes a tile of 8 x 32 cells: its 9 x 33 nodes are evaluated
// once into shared memory, then every thread writes its cell's 20 values
// contiguously.
constexpr int kFpRows = 8, kFpCols = 32;

template <typename T>
__device__ __forceinline__ void store_cell(T* dst, const T (&v)[20]) {
#pragma unroll
    for (int q = 0; q < 20; ++q) dst[q] = v[q];
}
template <>
__device__ __forceinline__ void store_cell<float>(float* dst, const float (&v)[20]) {
    float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int q = 0; q < 5; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

template <typename T>
__global__ void __launch_bounds__(256) field_prep(const double* __restrict__ phi, const double* __restrict__ Ec,
                                                  const double* __restrict__ Ess, const double* __restrict__ B, T* F,
                                                  T* rho, T* jm, int* sched, int NR, int nr, int i_win, int nnodes,
                                                  double dz, double dr, double cs, double sn, int magnetic,
                                                  TurnSet ts, HarmFields hf) {
    __shared__ T s_v[(kFpRows + 1) * (kFpCols + 1)][5];
    const int ci0 = blockIdx.y * kFpRows, cj0 = blockIdx.x * kFpCols;
    const int t = threadIdx.x;
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        if (t == 0) *sched = 0;     // the particle kernel's chunk counter
        // the step's Poisson solve: turn potentials at the next phase (the
        // coil nodes lie above the rows read here; set-up checks it) and
        // fresh refinement bookkeeping
        for (int q = t; q < ts.K; q += blockDim.x)
            ts.phi[ts.tn_node[q]] = turn_target(ts.st, nullptr, ts.tn_k[q], ts.nt, ts.cs, ts.sn);
        if (t < 2 * 16) ts.st->pnorm[t] = 0ull;
        if (t == 0) ts.st->pdone = 0;
    }
    for (int q = t; q < (kFpRows + 1) * (kFpCols + 1); q += blockDim.x) {
        const int i = ci0 + q / (kFpCols + 1), j = cj0 + q % (kFpCols + 1);
        if (i > i_win || j >= NR) continue;
        const int n = i * NR + j;
        // the step's deposits land on node rows 0..i_win only: clear them here
        // (each node by the tile that holds it as a lower-left node, the last
        // row and column by the tiles at the edge)
        const bool own = (q / (kFpCols + 1) < kFpRows || i == i_win) && (q % (kFpCols + 1) < kFpCols || j == NR - 1);
        if (own) {
            rho[n] = T(0);              // electrons
            rho[nnodes + n] = T(0);     // ions
            jm[n] = T(0);
        }
        double Ez = (i == 0) ? -(phi[n + NR] - phi[n]) / dz : -(phi[n + NR] - phi[n - NR]) / (2.0 * dz);
        double Er;
        if (j == 0) Er = 0.0;
        else if (j == NR - 1) Er = -(phi[n] - phi[n - 1]) / dr;
        else Er = -(phi[n + 1] - phi[n - 1]) / (2.0 * dr);
        // products and sums rounded separately (no contraction): the gather
        // fields then round to float exactly as the oracle's FP64 -> float32
        double Et = __dsub_rn(__dmul_rn(Ec[n], cs), __dmul_rn(Ess[n], sn));
        double Br = 0.0, Bz = 0.0;
        if (magnetic) {
            Br = __dadd_rn(__dmul_rn(B[n], cs), __dmul_rn(B[nnodes + n], sn));
            Bz = __dadd_rn(__dmul_rn(B[2 * nnodes + n], cs), __dmul_rn(B[3 * nnodes + n], sn));
        }
        // the retained harmonics, added in the order m = 2, 3, ...
        for (int h = 0; h < hf.ph.nh; ++h) {
            const double cm = hf.ph.c[h], sm = hf.ph.s[h];
            const double* E2 = hf.Ech + (size_t)h * 2 * nnodes;
            Et = __dadd_rn(Et, __dsub_rn(__dmul_rn(E2[n], cm), __dmul_rn(E2[nnodes + n], sm)));
            if (magnetic) {
                const double* B2 = hf.Bh + (size_t)h * 4 * nnodes;
                Br = __dadd_rn(Br, __dadd_rn(__dmul_rn(B2[n], cm), __dmul_rn(B2[nnodes + n], sm)));
                Bz = __dadd_rn(Bz, __dadd_rn(__dmul_rn(B2[2 * nnodes + n], cm), __dmul_rn(B2[3 * nnodes + n], sm)));
            }
        }
        s_v[q][0] = (T)Er;
        s_v[q][1] = (T)Ez;
        s_v[q][2] = (T)Et;
        s_v[q][3] = (T)Br;
        s_v[q][4] = (T)Bz;
    }
    __syncthreads();
    const int li = t / kFpCols, lj = t % kFpCols;
    const int ci = ci0 + li, cj = cj0 + lj;
    if (li >= kFpRows || ci >= i_win || cj >= nr) return;
    T v[20];
    // corners 00, 01, 10, 11 = nodes (ci, cj), (ci, cj+1), (ci+1, cj), (ci+1, cj+1)
    const int q00 = li * (kFpCols + 1) + lj;
    const int qs[4] = {q00, q00 + 1, q00 + kFpCols + 1, q00 + kFpCols + 2};
#pragma unroll
    for (int comp = 0; comp < 5; ++comp)
#pragma unroll
        for (int corner = 0; corner < 4; ++corner) v[comp * 4 + corner] = s_v[qs[corner]][comp];
    store_cell<T>(F + ((size_t)ci * nr + cj) * 20, v);
}

// ---------------------------------------------------------------- turn charge and accumulation
// Per step, one kernel: every thread adds its node's current harmonics
// (J_c += (2/N) cos(theta) J, J_s += (2/N) sin(theta) J, Eq. fourier, Kahan
// FP64), and one extra block takes the turn-charge sample: Q_k (Eq. facecharge)
// from the current phi, its harmonics, the trapezoid of Eq. pcap and the
// power sums, and advances the device step counter.
struct SampleArgs {
    DevState* st;
    const double* phi;
    const int* ft;
    const int* fnb;
    const int* fk;
    const double* fc;
    int nfaces, nt, n_rf;
    double cs, sn, two_over_n, inv_n;   // phase of the sample (after the step)
    const double* vol;
    double *Jc, *Js, *Jcc, *Jsc;
    int nn;
    double wc, ws;                      // (2/N) cos, (2/N) sin of the step's phase
    int* done;                          // the step's Poisson solve: final convergence decision
    int sweep;
    double tol;
    // retained harmonics: J harmonics (nh x 4 x nodes, with Kahan terms),
    // (2/N) cos m theta_old, (2/N) sin m theta_old, and cos m theta_new,
    // sin m theta_new of the charge sample
    double* Jh;
    int nnodes;
    HarmPhase wh, qh;
};

template <typename T>
__global__ void sample_accumulate(SampleArgs a, const T* jm) {
    // the last block takes the turn-charge sample alone, so its serial part
    // runs beside the node work of the other blocks
    if (blockIdx.x + 1 < gridDim.x) {
        int n = blockIdx.x * blockDim.x + threadIdx.x;
        if (n < a.nn) {
            double J = (double)jm[n] / a.vol[n];
            kahan_add(a.Jc[n], a.Jcc[n], a.wc * J);
            kahan_add(a.Js[n], a.Jsc[n], a.ws * J);
            for (int h = 0; h < a.wh.nh; ++h) {
                double* J4 = a.Jh + (size_t)h * 4 * a.nnodes;
                kahan_add(J4[n], J4[2 * a.nnodes + n], a.wh.c[h] * J);
                kahan_add(J4[a.nnodes + n], J4[3 * a.nnodes + n], a.wh.s[h] * J);
            }
        }
        return;
    }
    if (threadIdx.x == 0 && !*a.done) {
        DevState* s0 = a.st;
        double r = __longlong_as_double((long long)s0->pnorm[2 * a.sweep]);
        double sc = __longlong_as_double((long long)s0->pnorm[2 * a.sweep + 1]);
        double rel = (sc > 0) ? r / sc : 0.0;
        s0->prel = rel;
        s0->piters = a.sweep;
        if (rel <= a.tol) *a.done = 1;
        else s0->status |= PP_ST_NOCONV;
    }
    __shared__ double q[PP_MAX_TURNS];
    if (threadIdx.x < PP_MAX_TURNS) q[threadIdx.x] = 0;
    __syncthreads();
    for (int f = threadIdx.x; f < a.nfaces; f += blockDim.x)
        atomicAdd(&q[a.fk[f]], a.fc[f] * (a.phi[a.ft[f]] - a.phi[a.fnb[f]]));
    __syncthreads();
    if (threadIdx.x != 0) return;
    DevState* st = a.st;
    for (int k = 0; k < a.nt; ++k) {
        double V = turn_target(st, nullptr, k, a.nt, a.cs, a.sn);
        double Q = q[k];
        kahan_add(st->qc[k], st->qc_c[k], a.two_over_n * Q * a.cs);
        kahan_add(st->qs[k], st->qs_c[k], a.two_over_n * Q * a.sn);
        for (int h = 0; h < a.qh.nh; ++h) {
            kahan_add(st->qch[h][k], st->qchc[h][k], a.two_over_n * Q * a.qh.c[h]);
            kahan_add(st->qsh[h][k], st->qshc[h][k], a.two_over_n * Q * a.qh.s[h]);
        }
        if (st->n_samples == 0) {
            st->v_first[k] = V;
            st->q_first[k] = Q;
        } else {
            st->w[k] += 0.5 * (V + st->v_prev[k]) * (Q - st->q_prev[k]);
        }
        st->v_prev[k] = V;
        st->q_prev[k] = Q;
    }
    st->n_samples += 1;
    st->step += 1;
    kahan_add(st->p_ind, st->p_ind_c, st->p_ind_step * a.inv_n);
    kahan_add(st->p_es, st->p_es_c, st->p_es_step * a.inv_n);
    st->p_ind_step = 0;
    st->p_es_step = 0;
}

// ---------------------------------------------------------------- Helmholtz glue
__global__ void nodes_to_interior(const double* src, double* dst, int NZ, int NR, int j0, int M,
                                  double scale, const double* w) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int rows = NZ - 2;
    if (idx >= rows * M) return;
    int i = idx / M + 1, j = idx % M + j0;
    dst[idx] = scale * src[i * NR + j];
}

__global__ void interior_to_nodes(const double* src, double* dst, int NZ, int NR, int j0, int M) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= NZ * NR) return;
    int i = n / NR, j = n % NR;
    double v = 0.0;
    if (i >= 1 && i <= NZ - 2 && j >= j0 && j < j0 + M) v = src[(size_t)(i - 1) * M + (j - j0)];
    dst[n] = v;
}

void helmholtz_solve_sep(Cell* c, const SepSolver<double>& hs, const double* rhs_nodes, double* out_nodes,
                         double scale, cudaStream_t st) {
    int rows = hs.rows, M = hs.M;
    int nint = rows * M;
    double* stage = c->d_hstage;
    nodes_to_interior<<<(nint + 255) / 256, 256, 0, st>>>(rhs_nodes, stage, c->NZ, c->NR, 1, M, scale,
                                                           nullptr);
    sep_solve<double>(hs, stage, stage + nint, st, nullptr);
    interior_to_nodes<<<(c->nnodes + 255) / 256, 256, 0, st>>>(stage + nint, out_nodes, c->NZ, c->NR, 1, M);
    count_launch(2);
}

void helmholtz_solve_dev(Cell* c, const double* rhs_nodes, double* out_nodes, double scale,
                         cudaStream_t st) {
    helmholtz_solve_sep(c, c->hs, rhs_nodes, out_nodes, scale, st);
}

// ---------------------------------------------------------------- compose and B
// Eq. compose: E_c = E_c^(p) + sum I_s,k U_k, E_ss = E_ss^(p) + sum I_c,k U_k
// with I_k = I_c - i I_s (so I_s = -Im I_k, I_c = Re I_k).
__global__ void compose_kernel(const DevState* st, const double* x, double* Ec, double* Ess, double* Ecp,
                               double* Essp, const double* Ecp_new, const double* Essp_new, const double* U, int nn,
                               int nt, int use_new) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    if (use_new && st->accepted) {
        Ecp[n] = Ecp_new[n];
        Essp[n] = Essp_new[n];
    }
    double ec = Ecp[n], es = Essp[n];
    for (int k = 0; k < nt; ++k) {
        double ire = x[2 * (1 + k)], iim = x[2 * (1 + k) + 1];
        double u = U[(size_t)k * nn + n];
        ec += (-iim) * u;
        es += ire * u;
    }
    Ec[n] = ec;
    Ess[n] = es;
}

// B phasors from Faraday's law: B_r(t) = Brc cos + Brs sin with Brc = dEss/dz / w,
// Brs = dEc/dz / w; B_z(t) = Bzc cos + Bzs sin with Bzc = -(1/R) d(R Ess)/dR / w,
// Bzs = -(1/R) d(R Ec)/dR / w.
__global__ void bphasor_kernel(const double* Ec, const double* Ess, double* B, int NZ, int NR, double dz,
                               double dr, double omega) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    int nn = NZ * NR;
    if (n >= nn) return;
    int i = n / NR, j = n % NR;
    auto ddz = [&](const double* f) {
        if (i == 0) return (f[n + NR] - f[n]) / dz;
        if (i == NZ - 1) return (f[n] - f[n - NR]) / dz;
        return (f[n + NR] - f[n - NR]) / (2.0 * dz);
    };
    auto curl = [&](const double* f) {
        if (j == 0) return 2.0 * (f[n + 1] - f[n]) / dr;
        double R = j * dr;
        if (j == NR - 1) return __dsub_rn(__dmul_rn(R, f[n]), __dmul_rn(R - dr, f[n - 1])) / (dr * R);
        return __dsub_rn(__dmul_rn(R + dr, f[n + 1]), __dmul_rn(R - dr, f[n - 1])) / (2.0 * dr * R);
    };
    B[n] = ddz(Ess) / omega;
    B[nn + n] = ddz(Ec) / omega;
    B[2 * nn + n] = -curl(Ess) / omega;
    B[3 * nn + n] = -curl(Ec) / omega;
}

void launch_compose(Cell* c, bool from_new, cudaStream_t st) {
    int nn = c->nnodes;
    compose_kernel<<<(nn + 255) / 256, 256, 0, st>>>(c->d_st, c->d_st->x, c->d_Ec, c->d_Ess, c->d_Ecp, c->d_Essp,
                                                     c->d_Ecp_new, c->d_Essp_new, c->d_U, nn, c->nturns,
                                                     from_new ? 1 : 0);
    bphasor_kernel<<<(nn + 255) / 256, 256, 0, st>>>(c->d_Ec, c->d_Ess, c->d_Br, c->NZ, c->NR, c->dz, c->dr,
                                                     c->omega);
    count_launch(2);
    // the retained harmonics (Eq. compose and Faraday's law at m w)
    for (int h = 0; h + 1 < c->nharm; ++h) {
        double* E2 = c->d_Ech + (size_t)h * 2 * nn;
        double* P4 = c->d_Ecph + (size_t)h * 4 * nn;
        compose_kernel<<<(nn + 255) / 256, 256, 0, st>>>(c->d_st, c->d_st->xh[h], E2, E2 + nn, P4, P4 + nn,
                                                         P4 + 2 * nn, P4 + 3 * nn,
                                                         c->d_Uh + (size_t)h * c->nturns * nn, nn, c->nturns,
                                                         from_new ? 1 : 0);
        bphasor_kernel<<<(nn + 255) / 256, 256, 0, st>>>(E2, E2 + nn, c->d_Bh + (size_t)h * 4 * nn, c->NZ, c->NR,
                                                         c->dz, c->dr, (h + 2) * c->omega);
        count_launch(2);
    }
}

HarmPhase harm_phase(const Cell* c, double th) {
    HarmPhase p;
    p.nh = c->nharm - 1;
    for (int h = 0; h < kMaxHarm - 1; ++h) {
        p.c[h] = h < p.nh ? std::cos((h + 2) * th) : 0.0;
        p.s[h] = h < p.nh ? std::sin((h + 2) * th) : 0.0;
    }
    return p;
}

// ---------------------------------------------------------------- launchers
void launch_sample_accumulate(Cell* c, double th_old, double th_new, cudaStream_t st) {
    const double two_n = 2.0 / c->n_rf;
    const double cs_new = std::cos(th_new), sn_new = std::sin(th_new);
    const double wc = two_n * std::cos(th_old), ws = two_n * std::sin(th_old);
    SampleArgs a;
    a.st = c->d_st;
    a.phi = c->d_phi;
    a.ft = c->d_face_t;
    a.fnb = c->d_face_nb;
    a.fk = c->d_face_k;
    a.fc = c->d_face_c;
    a.nfaces = c->nfaces;
    a.nt = c->nturns;
    a.n_rf = c->n_rf;
    a.cs = cs_new;
    a.sn = sn_new;
    a.two_over_n = 2.0 / c->n_rf;
    a.inv_n = 1.0 / c->n_rf;
    a.vol = c->d_vol;
    a.Jc = c->d_Jc;
    a.Js = c->d_Js;
    a.Jcc = c->d_Jc_c;
    a.Jsc = c->d_Js_c;
    a.nn = (c->i_win + 1) * c->NR;
    a.wc = wc;
    a.ws = ws;
    a.done = &c->d_st->pdone;
    a.sweep = c->cfg.poisson_max_iter < 1 ? 1 : (c->cfg.poisson_max_iter > 15 ? 15 : c->cfg.poisson_max_iter);
    a.tol = c->cfg.poisson_tol;
    a.Jh = c->d_Jh;
    a.nnodes = c->nnodes;
    a.wh = harm_phase(c, th_old);
    for (int h = 0; h < a.wh.nh; ++h) {
        a.wh.c[h] *= two_n;
        a.wh.s[h] *= two_n;
    }
    a.qh = harm_phase(c, th_new);
    const unsigned nb = (unsigned)((a.nn + 255) / 256) + 1;     // + the sample block
    if (c->fp64)
        sample_accumulate<double><<<nb, 256, 0, st>>>(a, c->d_jm64);
    else
        sample_accumulate<float><<<nb, 256, 0, st>>>(a, c->d_jm);
    count_launch();
}

void launch_field_prep(Cell* c, double th, double th_next, cudaStream_t st) {
    const double cs = std::cos(th), sn = std::sin(th), cs_next = std::cos(th_next), sn_next = std::sin(th_next);
    dim3 grid((c->nr + kFpCols - 1) / kFpCols, (c->i_win + kFpRows - 1) / kFpRows);
    TurnSet ts{c->d_phi, c->d_tn_node, c->d_tn_k, c->ntn, c->nturns, c->d_st, cs_next, sn_next};
    HarmFields hf{c->d_Ech, c->d_Bh, harm_phase(c, th)};
    if (c->fp64)
        field_prep<double><<<grid, 256, 0, st>>>(c->d_phi, c->d_Ec, c->d_Ess, c->d_Br, c->d_F64, c->d_rho64, c->d_jm64,
                                                 &c->d_st->push_chunk, c->NR, c->nr, c->i_win, c->nnodes, c->dz, c->dr,
                                                 cs, sn, c->cfg.magnetic_force, ts, hf);
    else
        field_prep<float><<<grid, 256, 0, st>>>(c->d_phi, c->d_Ec, c->d_Ess, c->d_Br, c->d_F, c->d_rho, c->d_jm,
                                                &c->d_st->push_chunk, c->NR, c->nr, c->i_win, c->nnodes, c->dz, c->dr,
                                                cs, sn, c->cfg.magnetic_force, ts, hf);
    count_launch();
}

int poisson_refine(Cell* c, double cs, double sn, cudaStream_t st, bool external_targets,
                   const double* d_targets, bool in_step) {
    if (c->use_pcg) {
        // turn potentials and fresh bookkeeping (inside a step the field
        // preparation has imposed them already), then the persistent solve
        if (!in_step) {
            const int K = c->ntn;
            poisson_set_turns<<<(K + 63) / 64 > 0 ? (K + 63) / 64 : 1, 64, 0, st>>>(
                c->d_phi, c->d_tn_node, c->d_tn_k, K, c->d_st, external_targets ? d_targets : nullptr, c->nturns,
                cs, sn);
            count_launch();
        }
        return pcg_refine(c, cs, sn, st, external_targets ? d_targets : nullptr, in_step);
    }
    int rows = c->ps.rows, M = c->ps.M;
    int nint = rows * M;
    int maxit = c->cfg.poisson_max_iter < 1 ? 1 : (c->cfg.poisson_max_iter > 15 ? 15 : c->cfg.poisson_max_iter);
    // a solve outside a step (priming from zero, the period boundary's new
    // turn potentials, a standalone solve) has no previous step's potential
    // close to it: up to six sweeps (the converged ones are skipped on the device)
    if (!in_step && maxit < 6) maxit = 6;
    DevState* dst = c->d_st;
    int* done = &dst->pdone;
    const double* ext = external_targets ? d_targets : nullptr;
    PoisArgs a;
    a.phi = c->d_phi;
    a.rho = c->d_rho;
    a.rho_i = c->d_rho + c->nnodes;
    a.rho64 = c->fp64 ? c->d_rho64 : nullptr;
    a.rho64_i = c->fp64 ? c->d_rho64 + c->nnodes : nullptr;
    a.win = c->d_win;
    a.eps_row = c->d_eps_row;
    a.az = c->d_az;
    a.arp = c->d_arp;
    a.arm = c->d_arm;
    a.turn_mask = c->d_turn_mask;
    a.r32 = c->d_r32;
    a.NR = c->NR;
    a.NZ = c->NZ;
    a.M = M;
    a.inv2pieps0 = 1.0 / (2.0 * kPi * kEps0);
    a.done = done;
    a.st = dst;
    a.ext = ext;
    a.nt = c->nturns;
    a.cs = cs;
    a.sn = sn;
    const int K = c->ntn;
    if (!in_step) {
        poisson_set_turns<<<(K + 63) / 64 > 0 ? (K + 63) / 64 : 1, 64, 0, st>>>(c->d_phi, c->d_tn_node, c->d_tn_k, K,
                                                                               dst, ext, c->nturns, cs, sn);
        count_launch();
    }
    dim3 gblk(32, 8), ggrd((M + 31) / 32, (rows + 31) / 32);
    for (int it = 0; it <= maxit; ++it) {
        a.norm = &dst->pnorm[2 * it];
        poisson_residual<<<(nint + 255) / 256, 256, 0, st>>>(a);
        count_launch();
        if (it == maxit) {
            if (!in_step) {
                poisson_check<<<1, 32, 0, st>>>(dst, it, c->cfg.poisson_tol, done, 1);
                count_launch();
            }
            break;
        }
        // d0 = Vb-transform of the per-mode z solves of (r Vf)
        gemm_sweep<true><<<ggrd, gblk, 0, st>>>(c->d_r32, c->ps.Vf, c->ps.t0, rows, M, M, dst, it, c->cfg.poisson_tol,
                                                done);
        launch_pcr(c, c->ps.t0, c->ps.t1, st, done);
        gemm_sweep<false><<<ggrd, gblk, 0, st>>>(c->ps.t1, c->ps.Vb, c->ps.t0, rows, M, M, dst, it, 0.0, done);
        poisson_update_zt<<<(nint + 255) / 256, 256, 0, st>>>(c->d_phi, c->ps.t0, c->d_Zt, c->d_Ginv, c->d_tn_int, K,
                                                               c->ntn_pad, rows, M, c->NR, c->d_turn_mask, done);
        count_launch(4);
    }
    return 0;
}

// ---------------------------------------------------------------- allocation-free Poisson solve
// Scratch of pp_poisson_solve_noalloc: a fixed device array that lives as long
// as the library is loaded on each device that uses it, so the entry point
// itself never allocates.  Layout per call (bytes, each part 256-aligned):
// solver state | sigma (64 doubles) | zero charge (nnodes floats) |
// residual, transform and sweep buffers (3 x interior floats).
constexpr size_t kNoAllocBytes = (size_t)4 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void noalloc_report(const DevState* s, int* info) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        info[0] = s->piters + 1;
        info[1] = (s->status & PP_ST_NOCONV) ? 0 : 1;
    }
}

}  // namespace pp

#include <mutex>

namespace pp {
namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {nullptr};
}  // namespace
}  // namespace pp

extern "C" int pp_poisson_solve_noalloc(pp_cell* h, const double* d_q, const double* d_turn_phi, double* d_phi,
                                        int* d_info, void* stream) {
    using namespace pp;
    Cell* c = reinterpret_cast<Cell*>(h);
    if (!c || !d_q || !d_turn_phi || !d_phi) {
        set_error("bad argument to pp_poisson_solve_noalloc");
        return PP_E_ARG;
    }
    const int rows = c->ps.rows, M = c->ps.M, nint = rows * M;
    const size_t off_sig = align256(sizeof(DevState));
    const size_t off_rho = off_sig + align256(sizeof(double) * kMaxCapNodes);
    const size_t off_r32 = off_rho + align256(sizeof(float) * (size_t)c->nnodes);
    const size_t off_t0 = off_r32 + align256(sizeof(float) * (size_t)nint);
    const size_t off_t1 = off_t0 + align256(sizeof(float) * (size_t)nint);
    const size_t need = off_t1 + align256(sizeof(float) * (size_t)nint);
    if (need > kNoAllocBytes) {
        set_error("pp_poisson_solve_noalloc: grid needs " + std::to_string(need) + " bytes of scratch, the fixed "
                  "array holds " + std::to_string(kNoAllocBytes));
        return PP_E_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        set_error("pp_poisson_solve_noalloc: no usable current device");
        return PP_E_CUDA;
    }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                set_error(std::string("pp_poisson_solve_noalloc: cudaGetSymbolAddress failed: ") +
                          cudaGetErrorString(e));
                return PP_E_CUDA;
            }
            g_noalloc_addr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_noalloc_addr[dev]);
    }
    cudaStream_t st = (cudaStream_t)stream;
    DevState* sst = reinterpret_cast<DevState*>(base);
    double* sigma = reinterpret_cast<double*>(base + off_sig);
    float* rho0 = reinterpret_cast<float*>(base + off_rho);
    SepSolver<float> ps = c->ps;
    float* r32 = reinterpret_cast<float*>(base + off_r32);
    ps.t0 = reinterpret_cast<float*>(base + off_t0);
    ps.t1 = reinterpret_cast<float*>(base + off_t1);
    // what must start at zero: the solver state, the charge array the residual
    // adds to q, and the potential (its boundary values are the grounded zeros)
    cudaMemsetAsync(sst, 0, sizeof(DevState), st);
    cudaMemsetAsync(rho0, 0, sizeof(float) * (size_t)c->nnodes, st);
    cudaMemsetAsync(d_phi, 0, sizeof(double) * (size_t)c->nnodes, st);
    const int maxit = c->cfg.poisson_max_iter < 1 ? 1 : (c->cfg.poisson_max_iter > 15 ? 15 : c->cfg.poisson_max_iter);
    PoisArgs a;
    a.phi = d_phi;
    a.rho = rho0;
    a.rho_i = nullptr;
    a.rho64 = nullptr;
    a.rho64_i = nullptr;
    a.win = d_q;
    a.eps_row = c->d_eps_row;
    a.az = c->d_az;
    a.arp = c->d_arp;
    a.arm = c->d_arm;
    a.turn_mask = c->d_turn_mask;
    a.r32 = r32;
    a.NR = c->NR;
    a.NZ = c->NZ;
    a.M = M;
    a.inv2pieps0 = 1.0 / (2.0 * kPi * kEps0);
    a.done = &sst->pdone;
    a.st = sst;
    a.ext = d_turn_phi;
    a.nt = c->nturns;
    a.cs = 1.0;
    a.sn = 0.0;
    const int K = c->ntn;
    for (int it = 0; it <= maxit; ++it) {
        a.norm = &sst->pnorm[2 * it];
        poisson_residual<<<(nint + 255) / 256, 256, 0, st>>>(a);
        poisson_check<<<1, 32, 0, st>>>(sst, it, c->cfg.poisson_tol, &sst->pdone, it == maxit ? 1 : 0);
        count_launch(2);
        if (it == maxit) break;
        sep_solve<float>(ps, r32, ps.t0, st, &sst->pdone);
        poisson_cap<<<1, kMaxCapNodes, 0, st>>>(sst, d_turn_phi, d_phi, ps.t0, c->d_tn_node, c->d_tn_int, c->d_tn_k,
                                                c->d_Ginv, sigma, K, c->nturns, 1.0, 0.0, &sst->pdone);
        poisson_update<<<(nint + 255) / 256, 256, 0, st>>>(d_phi, ps.t0, c->d_Z, sigma, K, rows, M, c->NR,
                                                            c->d_turn_mask, sst, d_turn_phi, c->nturns, 1.0, 0.0,
                                                            &sst->pdone);
        count_launch(2);
    }
    if (d_info) {
        noalloc_report<<<1, 32, 0, st>>>(sst, d_info);
        count_launch();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("pp_poisson_solve_noalloc: ") + cudaGetErrorString(e));
        return PP_E_CUDA;
    }
    return PP_OK;
}

namespace pp {

// FP32 inner solve alone (used at initialisation for the capacitance columns)
void poisson_fast_solve(Cell* c, const float* rhs, float* out, cudaStream_t st) {
    sep_solve<float>(c->ps, rhs, out, st, nullptr);
}

}  // namespace pp
