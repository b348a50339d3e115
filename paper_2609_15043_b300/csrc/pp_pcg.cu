// The Poisson solve of the direct-implicit form (Sec. 2.3, Eq. poisson with the
// susceptibility chi, Eq. epseff) as one persistent thread-block cluster: FP64
// residual refinement around an FP32 preconditioned conjugate-gradient inner
// solve.
//
// chi(z, R) makes the operator non-separable.  The preconditioner is the
// separable operator with chi replaced by its mean over each node row,
// chibar(z) (the window slab and the plasma boundary at the electrode are then
// in the preconditioner; what is left is the radial profile of the plasma and
// particle noise): a radial transform, a per-mode tridiagonal solve in z by
// parallel cyclic reduction with coefficients formed on the fly from the rows'
// coupling and chibar, and the backward transform.  The turn nodes are
// Dirichlet nodes of the CG system, so the preconditioner is applied to the
// residual (zero there) and its result projected onto the free nodes (a
// principal block of a symmetric positive definite inverse).
//
// Layout: one cluster of up to 16 CTAs.  CTA c owns a band of interior rows
// (residual, vectors, stencil, transforms) and the modes m = c, c + C, ...
// (cyclic reduction).  Data crosses CTAs through global memory (L2); the
// phases are separated by a cluster barrier built from flags in distributed
// shared memory (release stores, acquire loads), every wait bounded: on
// expiry the barrier records PP_ST_TIMEOUT and the kernel runs to its end
// without further waiting.  The inner CG is the Chronopoulos-Gear form (both
// dot products of an iteration in one reduction), four barriers per
// iteration; dot products are reduced in a fixed order.  FP64 work (a small
// fraction of the FP32 rate on this part) is kept to the refinement residual
// and to single threads.
#include "pp_internal.h"

#include <cooperative_groups.h>
#include <string>
#include <vector>

namespace cg = cooperative_groups;

namespace pp {

namespace {

constexpr int kCT = 512;                  // threads per CTA
constexpr int kMaxC = 16;                 // CTAs of the cluster
constexpr int kMaxBand = 32;              // interior rows per CTA
constexpr int kEPT = 4;                   // cyclic-reduction rows per thread
constexpr int kMaxOuter = 6;              // FP64 refinement steps
constexpr int kMaxInner = 60;             // CG iterations per refinement step
constexpr double kInnerTol = 1e-6;        // inner residual reduction per refinement step at most (FP32)
constexpr int kAccN = 8;                  // partial sums per CTA

struct PcgArgs {
    double* phi;
    double* phi_prev;       // the previous step's potential (initial-guess extrapolation)
    int extrapolate;        // 1: start from 2 phi - phi_prev (inside a PIC step)
    const float* rho_e;
    const float* rho_i;
    const double* rho64_e;
    const double* rho64_i;
    const double* win;
    const double* chiw;
    double qm_e, qm_i;
    const signed char* turn_mask;
    int NR, M, rows, rows_pad;
    double inv2pieps0;
    const float* Vf;
    const float* Vb;
    const float* zlo;       // per interior row: eps_{i-1} / dz (z coupling below)
    const float* zup;       // eps_i / dz (above)
    const float* zeb;       // (dz / dR) (eps_{i-1} + eps_i) / 2 (radial weight)
    const float* mu;        // radial eigenvalues
    int L;                  // cyclic-reduction levels
    float* chib;            // chibar per node row
    const double* coef0;    // chi-free face coefficients per unknown (4, FP64, set-up)
    const float* coef0f;    // the same in FP32
    double* coef64;         // this solve's coefficients (Eq. epseff with chi), FP64
    float* coef32;          // the same in FP32 for the inner solve (vectors in global memory)
    float *rho, *z, *p, *s, *w, *dx;
    float* zl;              // the band's z when the vectors do not fit in shared memory
    float *rt, *st;         // rows x M transforms
    double* acc;            // [kMaxC][kAccN] partial sums
    DevState* dst;
    const double* ext;
    int nt;
    double cs, sn;
    double tol;
    size_t s_band_floats;   // floats of one band vector in shared memory (>= band rows x M, padded)
    int halo_nodes;         // nodes of the largest band's rows and two halo rows
    int sm_vec;             // 1: the CG vectors and FP32 coefficients live in shared memory
};

__device__ __forceinline__ double tgt_of(const DevState* st, const double* ext, int k, int nt, double cs,
                                         double sn) {
    if (ext) return ext[k];
    // Eq. dirichlet: phi_k = V_c cos + V_s sin with V = V_c - i V_s
    double vr = st->x[2 * (1 + nt + k)], vi = st->x[2 * (1 + nt + k) + 1];
    return vr * cs + (-vi) * sn;
}

// chi = (q_e/m_e rho_e + q_i/m_i rho_i) dt^2 / (eps0 V eps_r) (weights from set-up)
__device__ __forceinline__ double node_chi(const PcgArgs& a, int n) {
    const double wgt = a.chiw[n];
    if (wgt == 0.0) return 0.0;
    const double qe = a.rho64_e ? a.rho64_e[n] : (double)a.rho_e[n];
    const double qi = a.rho64_i ? a.rho64_i[n] : (double)a.rho_i[n];
    return wgt * (a.qm_e * qe + a.qm_i * qi);
}

__device__ __forceinline__ void st_release_cluster(unsigned* p, unsigned v) {
    asm volatile("st.release.cluster.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_cluster(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.cluster.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// barrier state in each CTA's shared memory: arrival words (used in CTA 0)
// and the release word
struct Bar {
    unsigned arrive[kMaxC];
    unsigned release;
    int ok;
};

// Cluster barrier: every CTA publishes its arrival in CTA 0 (release store),
// CTA 0 waits for all, then releases every CTA; waits are bounded.
__device__ __forceinline__ void cbar(Bar* b, unsigned& gen, int C, int rank, DevState* st) {
    __syncthreads();
    gen += 1;
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x == 0) {
        Bar* b0 = cl.map_shared_rank(b, 0);
        st_release_cluster(&b0->arrive[rank], gen);
    }
    if (rank == 0) {
        if ((int)threadIdx.x < C) {
            int it = 0;
            while (ld_acquire_cluster(&b->arrive[threadIdx.x]) != gen) {
                if (++it > (1 << 24)) {
                    atomicOr(&st->status, (unsigned)PP_ST_TIMEOUT);
                    b->ok = 0;
                    break;
                }
            }
        }
        __syncthreads();
        if ((int)threadIdx.x < C) st_release_cluster(&cl.map_shared_rank(b, (int)threadIdx.x)->release, gen);
    }
    if (threadIdx.x == 0) {
        int it = 0;
        while (ld_acquire_cluster(&b->release) != gen) {
            if (++it > (1 << 24)) {
                atomicOr(&st->status, (unsigned)PP_ST_TIMEOUT);
                b->ok = 0;
                break;
            }
        }
    }
    __syncthreads();
}

// Block reduction: the warps reduce in FP32, one thread combines the warps'
// partials in FP64; the result is broadcast through shared memory.
__device__ __forceinline__ double block_reduce(float v, bool mx, float* red, double* bc) {
    for (int o = 16; o > 0; o >>= 1) {
        const float u = __shfl_xor_sync(0xffffffffu, v, o);
        v = mx ? fmaxf(v, u) : v + u;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = mx ? fmax(t, (double)red[q]) : t + (double)red[q];
        bc[0] = t;
    }
    __syncthreads();
    return bc[0];
}

// sum / max of the C per-CTA partials of a slot: warp 0 loads them in
// parallel (one memory latency) and reduces, the block reads the broadcast
__device__ __forceinline__ double cta_reduce(const double* acc, int C, int slot, bool mx, double* bc) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double v = lane < C ? __ldcg(acc + (size_t)lane * kAccN + slot) : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_xor_sync(0xffffffffu, v, o);
            v = mx ? fmax(v, u) : v + u;
        }
        if (lane == 0) bc[1] = v;
    }
    __syncthreads();
    const double r = bc[1];
    __syncthreads();
    return r;
}

// s_out (nr x Mp) = in (nr x M, 16-byte aligned rows) * V: a thread owns a
// 4 x 4 tile (four rows, one column quad) over a slice of k, reading four k
// of a row as one float4 and V's rows as float4 quads; the slices' partial
// tiles are added in shared memory.  M is a multiple of 4.
__device__ void transform(const float* in, int nr, const float* __restrict__ V, int M, float* s_out) {
    const int Mp = (M + 31) & ~31;
    const int nq = M / 4, nrc = (nr + 3) / 4;
    const int per_g = nq * nrc;
    int G = kCT / per_g;
    G = max(1, min(G, M / 8));
    const int kc = (((M + G - 1) / G) + 3) & ~3;
    for (int q = threadIdx.x; q < nr * Mp; q += kCT) s_out[q] = 0.f;
    __syncthreads();
    const int t = threadIdx.x;
    const int g = t / per_g, rest = t % per_g;
    const int rc = rest / nq, cq = rest % nq;
    if (g < G) {
        const int k0 = g * kc, k1 = min(M, k0 + kc);
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
        const float4* V4 = reinterpret_cast<const float4*>(V);
        for (int k = k0; k < k1; k += 4) {
            const float4 v0 = __ldg(V4 + (size_t)(k + 0) * nq + cq);
            const float4 v1 = __ldg(V4 + (size_t)(k + 1) * nq + cq);
            const float4 v2 = __ldg(V4 + (size_t)(k + 2) * nq + cq);
            const float4 v3 = __ldg(V4 + (size_t)(k + 3) * nq + cq);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = rc * 4 + r;
                if (row < nr) {
                    const float4 x = *reinterpret_cast<const float4*>(in + (size_t)row * M + k);
                    acc[r][0] = fmaf(x.x, v0.x, fmaf(x.y, v1.x, fmaf(x.z, v2.x, fmaf(x.w, v3.x, acc[r][0]))));
                    acc[r][1] = fmaf(x.x, v0.y, fmaf(x.y, v1.y, fmaf(x.z, v2.y, fmaf(x.w, v3.y, acc[r][1]))));
                    acc[r][2] = fmaf(x.x, v0.z, fmaf(x.y, v1.z, fmaf(x.z, v2.z, fmaf(x.w, v3.z, acc[r][2]))));
                    acc[r][3] = fmaf(x.x, v0.w, fmaf(x.y, v1.w, fmaf(x.z, v2.w, fmaf(x.w, v3.w, acc[r][3]))));
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int row = rc * 4 + r;
            if (row < nr)
#pragma unroll
                for (int c = 0; c < 4; ++c) atomicAdd(&s_out[row * Mp + 4 * cq + c], acc[r][c]);
        }
    }
    __syncthreads();
}

// Per-mode tridiagonal solves in z of the CTA's modes by parallel cyclic
// reduction, the coefficients formed from the rows' couplings and chibar:
// a_i = zlo_i f(i, i-1), c_i = zup_i f(i, i+1), b_i = -(zlo_i f(i, i-1) +
// zup_i f(i, i+1)) + zeb_i (1 + chibar_i) mu_m with f(i, k) = 1 + (chibar_i +
// chibar_k) / 2; passes of P = kCT / (rows_pad / kEPT) modes.
__device__ void pcr_modes(const PcgArgs& a, int rank, int C, float* sh) {
    const int rows = a.rows, M = a.M, L = a.L, rp = a.rows_pad;
    const int Tm = rp / kEPT;
    const int P = kCT / Tm;
    const int nmodes = (M - rank + C - 1) / C;
    const size_t bs = (size_t)P * rp;             // one coefficient array of a pass
    auto buf = [&](int q, int v) { return sh + (size_t)(q * 5 + v) * bs; };   // a, b, 1/b, c, d
    for (int base = 0; base < nmodes; base += P) {
        const int lm = threadIdx.x / Tm, e = threadIdx.x % Tm;
        const int mi = base + lm;
        const bool act = mi < nmodes;
        const int m = rank + mi * C;
        const float mum = act ? __ldg(a.mu + m) : 0.f;
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            const int i = e + k * Tm;
            float av = 0.f, bv = 1.f, cv = 0.f, dv = 0.f;
            if (act && i < rows) {
                const float ch = __ldcg(a.chib + i + 1);
                const float flo = 1.f + 0.5f * (ch + __ldcg(a.chib + i));
                const float fup = 1.f + 0.5f * (ch + __ldcg(a.chib + i + 2));
                const float lo = __ldg(a.zlo + i) * flo, up = __ldg(a.zup + i) * fup;
                av = i > 0 ? lo : 0.f;
                cv = i + 1 < rows ? up : 0.f;
                bv = fmaf(__ldg(a.zeb + i) * (1.f + ch), mum, -(lo + up));
                dv = __ldcg(a.rt + (size_t)i * M + m);
            }
            const int q = lm * rp + i;
            buf(0, 0)[q] = av;
            buf(0, 1)[q] = bv;
            buf(0, 2)[q] = __frcp_rn(bv);
            buf(0, 3)[q] = cv;
            buf(0, 4)[q] = dv;
        }
        __syncthreads();
        // each row's b is a divisor of both neighbours at a level: its
        // reciprocal is formed once per row and level
        int cur = 0;
        for (int l = 0; l < L; ++l) {
            const int stp = 1 << l;
            const float* A = buf(cur, 0) + lm * rp;
            const float* B = buf(cur, 1) + lm * rp;
            const float* IB = buf(cur, 2) + lm * rp;
            const float* Cc = buf(cur, 3) + lm * rp;
            const float* D = buf(cur, 4) + lm * rp;
            float* A2 = buf(cur ^ 1, 0) + lm * rp;
            float* B2 = buf(cur ^ 1, 1) + lm * rp;
            float* IB2 = buf(cur ^ 1, 2) + lm * rp;
            float* C2 = buf(cur ^ 1, 3) + lm * rp;
            float* D2 = buf(cur ^ 1, 4) + lm * rp;
#pragma unroll
            for (int k = 0; k < kEPT; ++k) {
                const int i = e + k * Tm;
                if (i < rows) {
                    const int im = i - stp, ip = i + stp;
                    float b2 = B[i], d2 = D[i], a2 = 0.f, c2 = 0.f;
                    if (im >= 0) {
                        const float al = -A[i] * IB[im];
                        a2 = al * A[im];
                        b2 = fmaf(al, Cc[im], b2);
                        d2 = fmaf(al, D[im], d2);
                    }
                    if (ip < rows) {
                        const float ga = -Cc[i] * IB[ip];
                        c2 = ga * Cc[ip];
                        b2 = fmaf(ga, A[ip], b2);
                        d2 = fmaf(ga, D[ip], d2);
                    }
                    A2[i] = a2;
                    B2[i] = b2;
                    IB2[i] = __frcp_rn(b2);
                    C2[i] = c2;
                    D2[i] = d2;
                }
            }
            __syncthreads();
            cur ^= 1;
        }
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            const int i = e + k * Tm;
            if (act && i < rows) {
                const int q = lm * rp + i;
                a.st[(size_t)i * M + m] = buf(cur, 4)[q] * buf(cur, 2)[q];
            }
        }
        __syncthreads();
    }
}

}  // namespace

__global__ void __launch_bounds__(kCT, 1) pcg_cluster(PcgArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Bar bar;
    __shared__ float red[kCT / 32];
    __shared__ double bc[4];

    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int C = (int)cl.num_blocks();
    const int M = a.M, NR = a.NR;
    const int lo = (int)((long long)a.rows * rank / C), hi = (int)((long long)a.rows * (rank + 1) / C);
    const int nb = hi - lo, nbM = nb * M;
    const size_t band = a.s_band_floats;
    // shared layout: chi of the band's node rows and their two halo rows
    // (FP64), transform staging and accumulation, cyclic-reduction buffers,
    // the free-node mask, and (when they fit) the CG vectors and the FP32
    // face coefficients of the band
    double* s_chi = reinterpret_cast<double*>(smem);
    float* s_in = reinterpret_cast<float*>(s_chi + a.halo_nodes);
    float* s_out = s_in + band;
    float* s_pcr = s_out + band;
    unsigned char* s_free = reinterpret_cast<unsigned char*>(s_pcr + 10 * (size_t)kCT * kEPT);
    float* vec = reinterpret_cast<float*>(s_free + band);
    float *R, *DX, *P, *S, *W, *Z, *CF;
    if (a.sm_vec) {
        R = vec;
        DX = vec + band;
        P = vec + 2 * band;
        S = vec + 3 * band;
        W = vec + 4 * band;
        Z = vec + 5 * band;
        CF = vec + 6 * band;
    } else {
        const size_t o = (size_t)lo * M;
        R = a.rho + o;
        DX = a.dx + o;
        P = a.p + o;
        S = a.s + o;
        W = a.w + o;
        Z = a.zl + o;
        CF = a.coef32 + 4 * o;
    }
    if (threadIdx.x < kMaxC) bar.arrive[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
        bar.release = 0u;
        bar.ok = 1;
    }
    unsigned gen = 0;
    cl.sync();                                     // every CTA's barrier words initialised
    double* my_acc = a.acc + (size_t)rank * kAccN;
    auto all_sum = [&](int slot) { return cta_reduce(a.acc, C, slot, false, bc); };
    auto all_max = [&](int slot) { return cta_reduce(a.acc, C, slot, true, bc); };

    // node rows lo .. hi + 1 (the band's interior rows and one halo row on
    // each side) are contiguous in the node grid
    const int hn = (nb + 2) * NR;
    const size_t n0 = (size_t)lo * NR;
    for (int q = threadIdx.x; q < hn; q += kCT) s_chi[q] = node_chi(a, (int)(n0 + q));
    for (int li = threadIdx.x; li < nbM; li += kCT)
        s_free[li] = a.turn_mask[(lo + li / M + 1) * NR + li % M] < 0 ? 1 : 0;
    __syncthreads();
    // chibar of the band's node rows (and of the electrode and lid rows at the
    // ends of the cluster): the mean of chi over the interior columns
    for (int r = threadIdx.x; r < nb + 2; r += kCT) {
        const bool own = (r >= 1 && r <= nb) || (r == 0 && rank == 0) || (r == nb + 1 && rank == C - 1);
        if (own) {
            double t = 0.0;
            for (int j = 0; j < M; ++j) t += s_chi[r * NR + j];
            a.chib[lo + r] = (float)(t / M);
        }
    }
    // initial guess inside a step: 2 phi - phi_prev on the free nodes
    if (a.extrapolate) {
        const bool have = a.dst->phi_prev_ok != 0;
        for (int li = threadIdx.x; li < nbM; li += kCT) {
            if (!s_free[li]) continue;
            const size_t n = (size_t)(lo + li / M + 1) * NR + li % M;
            const double pc = a.phi[n];
            if (have) a.phi[n] = 2.0 * pc - a.phi_prev[n];
            a.phi_prev[n] = pc;
        }
        cbar(&bar, gen, C, rank, a.dst);
    }

    double rel = 0.0, scale = 0.0;
    bool conv = false;
    int inner_total = 0, outer = 0;
    for (;; ++outer) {
        // ---- FP64 residual r = b - A phi on the band (slot 0: max |r|, slot
        // 1: the componentwise scale of the first pass); the face coefficients
        // are the set-up's chi-free ones times the factor of Eq. epseff
        double rmax = 0.0, smax = 0.0;
        for (int li = threadIdx.x; li < nbM; li += kCT) {
            const int ii = li / M, j = li % M;
            const int i = lo + ii + 1;
            const int n = i * NR + j;
            const size_t gi = (size_t)4 * (lo * M + li);
            double c0, c1, c2, c3;
            if (outer == 0) {
                const int sn = (ii + 1) * NR + j;
                const double xc = s_chi[sn];
                c0 = a.coef0[gi] * (1.0 + 0.5 * (xc + s_chi[sn + NR]));
                c1 = a.coef0[gi + 1] * (1.0 + 0.5 * (xc + s_chi[sn - NR]));
                c2 = a.coef0[gi + 2] * (1.0 + 0.5 * (xc + s_chi[sn + 1]));
                c3 = j > 0 ? a.coef0[gi + 3] * (1.0 + 0.5 * (xc + s_chi[sn - 1])) : 0.0;
                a.coef64[gi] = c0;
                a.coef64[gi + 1] = c1;
                a.coef64[gi + 2] = c2;
                a.coef64[gi + 3] = c3;
                const float xf = (float)xc;
                CF[4 * li] = a.coef0f[gi] * (1.f + 0.5f * (xf + (float)s_chi[sn + NR]));
                CF[4 * li + 1] = a.coef0f[gi + 1] * (1.f + 0.5f * (xf + (float)s_chi[sn - NR]));
                CF[4 * li + 2] = a.coef0f[gi + 2] * (1.f + 0.5f * (xf + (float)s_chi[sn + 1]));
                CF[4 * li + 3] = j > 0 ? a.coef0f[gi + 3] * (1.f + 0.5f * (xf + (float)s_chi[sn - 1])) : 0.f;
            } else {
                c0 = a.coef64[gi];
                c1 = a.coef64[gi + 1];
                c2 = a.coef64[gi + 2];
                c3 = a.coef64[gi + 3];
            }
            float rv = 0.f;
            const double pc = a.phi[n];
            if (!s_free[li]) {
                const double diag = c0 + c1 + c2 + c3;
                const double tg = tgt_of(a.dst, a.ext, a.turn_mask[n], a.nt, a.cs, a.sn);
                rmax = fmax(rmax, fabs(tg - pc) * diag);
                if (outer == 0) smax = fmax(smax, fabs(tg) * diag);
            } else {
                const double pu = a.phi[n + NR], pd = a.phi[n - NR], pr = a.phi[n + 1];
                const double pl = j > 0 ? a.phi[n - 1] : pc;
                const double qe = a.rho64_e ? a.rho64_e[n] : (double)a.rho_e[n];
                const double qi = a.rho64_e ? a.rho64_i[n] : (double)a.rho_i[n];
                const double b = -((qe + qi) + a.win[n]) * a.inv2pieps0;
                // b - sum_f c_f (phi_f - phi_c) in fused form
                const double ap = fma(c3, pl - pc, fma(c2, pr - pc, fma(c1, pd - pc, c0 * (pu - pc))));
                const double r = b - ap;
                rmax = fmax(rmax, fabs(r));
                if (outer == 0)
                    smax = fmax(smax, fabs(b) + fabs(c0 * (pu - pc)) + fabs(c1 * (pd - pc)) + fabs(c2 * (pr - pc)) +
                                          fabs(c3 * (pl - pc)));
                // inner system B dx = -r with B = -A (positive definite)
                rv = (float)(-r);
            }
            R[li] = rv;
            DX[li] = 0.f;
        }
        rmax = block_reduce((float)rmax, true, red, bc);
        if (outer == 0) smax = block_reduce((float)smax, true, red, bc);
        if (threadIdx.x == 0) {
            my_acc[0] = rmax;
            if (outer == 0) my_acc[1] = smax;
        }
        cbar(&bar, gen, C, rank, a.dst);
        if (outer == 0) scale = all_max(1);
        rel = scale > 0 ? all_max(0) / scale : 0.0;
        conv = rel <= a.tol;
        if (conv || outer == kMaxOuter || !bar.ok) break;

        // ---- inner CG (Chronopoulos-Gear) on B dx = rho with the projected
        // chibar preconditioner z = -(Pi P_chibar Pi rho)
        double gam = 0.0, alpha = 0.0, beta = 0.0, r0 = 0.0;
        for (int it = 0;; ++it) {
            // (A) update (it > 0), max |rho|, forward transform
            float rmf = 0.f;
            const float alf = (float)alpha;
            for (int li = threadIdx.x; li < nbM; li += kCT) {
                float rv = R[li];
                if (it > 0 && s_free[li]) {
                    DX[li] = fmaf(alf, P[li], DX[li]);
                    rv = fmaf(-alf, S[li], rv);
                    R[li] = rv;
                }
                rmf = fmaxf(rmf, fabsf(rv));
            }
            const double rm = block_reduce(rmf, true, red, bc);
            if (threadIdx.x == 0) my_acc[2] = rm;
            transform(R, nb, a.Vf, M, s_out);
            {
                const int Mp = (M + 31) & ~31;
                for (int q = threadIdx.x; q < nbM; q += kCT) a.rt[(size_t)lo * M + q] = s_out[(q / M) * Mp + q % M];
            }
            cbar(&bar, gen, C, rank, a.dst);
            // (B) convergence of the inner solve, cyclic reduction
            // the inner solve stops at half the refinement's target residual
            // (in absolute terms, so a good initial guess saves iterations),
            // or at the reduction FP32 can deliver
            const double rn = all_max(2);
            if (it == 0) r0 = rn;
            if (!bar.ok || rn <= fmax(0.5 * a.tol * scale, kInnerTol * r0) || it == kMaxInner) break;
            pcr_modes(a, rank, C, s_pcr);
            cbar(&bar, gen, C, rank, a.dst);
            // (C) backward transform of the band, projected onto the free
            // nodes: z = -(P rho); the band of z is published for the
            // neighbours' stencils
            for (int q = threadIdx.x; q < nbM; q += kCT) s_in[q] = __ldcg(a.st + (size_t)lo * M + q);
            __syncthreads();
            transform(s_in, nb, a.Vb, M, s_out);
            {
                const int Mp = (M + 31) & ~31;
                for (int li = threadIdx.x; li < nbM; li += kCT) {
                    const float zv = s_free[li] ? -s_out[(li / M) * Mp + li % M] : 0.f;
                    Z[li] = zv;
                    a.z[(size_t)lo * M + li] = zv;
                }
            }
            cbar(&bar, gen, C, rank, a.dst);
            // (D) w = B z on the band (halo rows of z from the neighbours),
            // gamma = rho . z, delta = z . w
            float pgf = 0.f, pdf = 0.f;
            for (int li = threadIdx.x; li < nbM; li += kCT) {
                float wv = 0.f;
                const float zc = Z[li];
                if (s_free[li]) {
                    const int ii = li / M, j = li % M;
                    const int gi = lo + ii;
                    const float* c = CF + 4 * li;
                    const float zu = ii + 1 < nb ? Z[li + M] : (gi + 1 < a.rows ? __ldcg(a.z + (size_t)(gi + 1) * M + j) : 0.f);
                    const float zd = ii > 0 ? Z[li - M] : (gi > 0 ? __ldcg(a.z + (size_t)(gi - 1) * M + j) : 0.f);
                    const float zr = j + 1 < M ? Z[li + 1] : 0.f;
                    const float zlf = j > 0 ? Z[li - 1] : 0.f;
                    float y = c[0] * (zu - zc) + c[1] * (zd - zc) + c[2] * (zr - zc);
                    if (j > 0) y += c[3] * (zlf - zc);
                    wv = -y;
                }
                W[li] = wv;
                pgf = fmaf(R[li], zc, pgf);
                pdf = fmaf(zc, wv, pdf);
            }
            const double pg = block_reduce(pgf, false, red, bc);
            const double pd = block_reduce(pdf, false, red, bc);
            if (threadIdx.x == 0) {
                my_acc[3] = pg;
                my_acc[4] = pd;
            }
            cbar(&bar, gen, C, rank, a.dst);
            // (E) the scalars (one thread) and the new directions
            const double gn = all_sum(3), dn = all_sum(4);
            if (threadIdx.x == 0) {
                double al, be;
                if (it == 0) {
                    be = 0.0;
                    al = dn > 0 ? gn / dn : 0.0;
                } else {
                    be = gam != 0.0 ? gn / gam : 0.0;
                    const double den = dn - be * gn / alpha;
                    al = den > 0 ? gn / den : 0.0;
                }
                bc[2] = al;
                bc[3] = be;
            }
            __syncthreads();
            alpha = bc[2];
            beta = bc[3];
            gam = gn;
            const float bef = (float)beta;
            for (int li = threadIdx.x; li < nbM; li += kCT) {
                const float zv = Z[li], wv = W[li];
                P[li] = it == 0 ? zv : fmaf(bef, P[li], zv);
                S[li] = it == 0 ? wv : fmaf(bef, S[li], wv);
            }
            ++inner_total;
        }
        // phi += dx on the free nodes of the band; the next residual reads the
        // neighbours' rows after the barrier
        for (int li = threadIdx.x; li < nbM; li += kCT)
            if (s_free[li]) a.phi[(size_t)(lo + li / M + 1) * NR + li % M] += (double)DX[li];
        cbar(&bar, gen, C, rank, a.dst);
        if (!bar.ok) break;
    }
    if (rank == 0 && threadIdx.x == 0) {
        DevState* st = a.dst;
        st->prel = rel;
        st->piters = inner_total + outer;
        st->pdone = 1;
        if (a.extrapolate) st->phi_prev_ok = 1;
        if (!conv) st->status |= PP_ST_NOCONV;
    }
    cl.sync();                                     // no CTA leaves while others may write its flags
}

// ---------------------------------------------------------------- host side
namespace {
size_t pcg_smem(const Cell* c, int C, size_t* band, int* halo, int* sm_vec) {
    const int M = c->ps.M, rows = c->ps.rows;
    const int nbmax = (rows + C - 1) / C;
    const int Mp = (M + 31) & ~31;
    size_t bf = (size_t)nbmax * Mp;
    bf = (bf + 15) & ~(size_t)15;
    *band = bf;
    *halo = ((nbmax + 2) * c->NR + 1) & ~1;
    const size_t base = sizeof(double) * (size_t)(*halo) + sizeof(float) * (2 * bf + 10 * (size_t)kCT * kEPT) + bf;
    const size_t with_vec = base + sizeof(float) * 10 * bf;
    *sm_vec = with_vec <= (size_t)200 * 1024 ? 1 : 0;
    return *sm_vec ? with_vec : base;
}

// 16 CTAs when the device schedules such clusters (non-portable size) with
// the cell's shared memory, else 8
int pcg_cluster_size(const Cell* c) {
    int C = 16;
    if (cudaFuncSetAttribute(pcg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) C = 8;
    cudaGetLastError();
    for (; C >= 8; C /= 2) {
        size_t band = 0;
        int halo = 0, smv = 0;
        const size_t shm = pcg_smem(c, C, &band, &halo, &smv);
        if (cudaFuncSetAttribute(pcg_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3(kCT);
        cfg.dynamicSmemBytes = shm;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, pcg_cluster, &cfg) == cudaSuccess && n > 0) return C;
        cudaGetLastError();
    }
    return 0;
}
}  // namespace

int pcg_supported(Cell* c) {
    const int rows = c->ps.rows, M = c->ps.M;
    int rows_pad = 1;
    while (rows_pad < rows) rows_pad <<= 1;
    if (rows_pad < kEPT) rows_pad = kEPT;
    if (!(M <= kCT && M % 4 == 0 && rows <= 1024 && rows_pad / kEPT <= kCT && c->pcr_levels <= kMaxPcrLevels))
        return 0;
    const int C = pcg_cluster_size(c);
    if (C < 8 || (rows + C - 1) / C > kMaxBand) return 0;
    c->pcg_blocks = C;
    return 1;
}

void pcg_alloc(Cell* c, const std::vector<double>& az, const std::vector<double>& arp,
               const std::vector<double>& arm, const std::vector<double>& mu) {
    const int M = c->ps.M, rows = c->ps.rows;
    const size_t nint = (size_t)rows * M;
    // the chi-free face coefficients of every interior unknown (z+, z-, R+, R-),
    // the Poisson operator divided by 2 pi (Eq. epseff with chi = 0, Eq. areas)
    {
        std::vector<double> cf(nint * 4);
        std::vector<float> cff(nint * 4);
        for (size_t idx = 0; idx < nint; ++idx) {
            const int i = (int)(idx / M) + 1, j = (int)(idx % M);
            const double epz = c->eps_row[i], emz = c->eps_row[i - 1], eb = 0.5 * (emz + epz);
            const double v[4] = {az[j] * epz, az[j] * emz, eb * arp[j], j > 0 ? eb * arm[j] : 0.0};
            for (int f = 0; f < 4; ++f) {
                cf[4 * idx + f] = v[f];
                cff[4 * idx + f] = (float)v[f];
            }
        }
        c->d_pcg0 = c->alloc<double>(nint * 4);
        c->d_pcg0f = c->alloc<float>(nint * 4);
        cudaMemcpy(c->d_pcg0, cf.data(), sizeof(double) * nint * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_pcg0f, cff.data(), sizeof(float) * nint * 4, cudaMemcpyHostToDevice);
    }
    // the rows' couplings of the per-mode z systems (as in the separable
    // solver) and the radial eigenvalues
    {
        std::vector<float> zr((size_t)3 * rows), mf(M);
        for (int ii = 0; ii < rows; ++ii) {
            const int i = ii + 1;
            const double ep = c->eps_row[i], em = c->eps_row[i - 1];
            zr[ii] = (float)(em / c->dz);
            zr[rows + ii] = (float)(ep / c->dz);
            zr[2 * rows + ii] = (float)((c->dz / c->dr) * 0.5 * (ep + em));
        }
        for (int m = 0; m < M; ++m) mf[m] = (float)mu[m];
        c->d_pcg_zrow = c->alloc<float>((size_t)3 * rows);
        c->d_pcg_mu = c->alloc<float>(M);
        cudaMemcpy(c->d_pcg_zrow, zr.data(), sizeof(float) * 3 * rows, cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_pcg_mu, mf.data(), sizeof(float) * M, cudaMemcpyHostToDevice);
    }
    c->d_pcg = c->alloc<double>(nint * 4);               // this solve's FP64 face coefficients
    c->d_pcg32 = c->alloc<float>(nint * 10);             // FP32 coefficients (4), rho, z, p, s, w, dx
    c->d_pcg_acc = c->alloc<double>((size_t)kMaxC * kAccN);
    c->d_pcg_chib = c->alloc<float>((size_t)c->NZ + 2);
    c->d_phi_prev = c->alloc<double>(c->nnodes);
}

int pcg_refine(Cell* c, double cs, double sn, cudaStream_t st, const double* ext, bool in_step) {
    const size_t nint = (size_t)c->ps.rows * c->ps.M;
    const int C = c->pcg_blocks;                  // the cluster size chosen at set-up
    PcgArgs a;
    a.phi = c->d_phi;
    a.phi_prev = c->d_phi_prev;
    a.extrapolate = in_step ? 1 : 0;
    if (c->fp64) {
        a.rho_e = a.rho_i = nullptr;
        a.rho64_e = c->d_rho64;
        a.rho64_i = c->d_rho64 + c->nnodes;
    } else {
        a.rho_e = c->d_rho;
        a.rho_i = c->d_rho + c->nnodes;
        a.rho64_e = a.rho64_i = nullptr;
    }
    a.win = c->d_win;
    a.chiw = c->d_chiw;
    a.qm_e = c->chi_qm[0];
    a.qm_i = c->chi_qm[1];
    a.turn_mask = c->d_turn_mask;
    a.NR = c->NR;
    a.M = c->ps.M;
    a.rows = c->ps.rows;
    int rp = 1;
    while (rp < a.rows) rp <<= 1;
    if (rp < kEPT) rp = kEPT;
    a.rows_pad = rp;
    a.inv2pieps0 = 1.0 / (2.0 * kPi * kEps0);
    a.Vf = c->ps.Vf;
    a.Vb = c->ps.Vb;
    a.zlo = c->d_pcg_zrow;
    a.zup = c->d_pcg_zrow + a.rows;
    a.zeb = c->d_pcg_zrow + 2 * a.rows;
    a.mu = c->d_pcg_mu;
    a.L = c->pcr_levels;
    a.chib = c->d_pcg_chib;
    a.coef0 = c->d_pcg0;
    a.coef0f = c->d_pcg0f;
    a.coef64 = c->d_pcg;
    a.coef32 = c->d_pcg32;
    a.rho = c->d_pcg32 + 4 * nint;
    a.z = c->d_pcg32 + 5 * nint;
    a.p = c->d_pcg32 + 6 * nint;
    a.s = c->d_pcg32 + 7 * nint;
    a.w = c->d_pcg32 + 8 * nint;
    a.dx = c->d_pcg32 + 9 * nint;
    a.zl = a.z;
    a.rt = c->ps.t0;
    a.st = c->ps.t1;
    a.acc = c->d_pcg_acc;
    a.dst = c->d_st;
    a.ext = ext;
    a.nt = c->nturns;
    a.cs = cs;
    a.sn = sn;
    a.tol = c->cfg.poisson_tol;
    size_t band = 0;
    int halo = 0, smv = 0;
    const size_t shm = pcg_smem(c, C, &band, &halo, &smv);
    a.s_band_floats = band;
    a.halo_nodes = halo;
    a.sm_vec = smv;
    cudaFuncSetAttribute(pcg_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = shm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, pcg_cluster, a);
    count_launch();
    if (e != cudaSuccess) {
        set_error(std::string("Poisson cluster launch: ") + cudaGetErrorString(e));
        return PP_E_CUDA;
    }
    return 0;
}

}  // namespace pp
