// The Poisson solve of the direct-implicit form (Sec. 2.3, Eq. poisson with the
// susceptibility chi, Eq. epseff) as one persistent thread-block cluster: FP64
// residual refinement around an FP32 preconditioned conjugate-gradient inner
// solve.
//
// chi(z, R) makes the operator non-separable.  The preconditioner is the
// separable operator with chi replaced by its mean over each node row,
// chibar(z) (the window slab and the plasma boundary at the electrode are then
// in the preconditioner; what is left is the radial profile of the plasma and
// particle noise): a radial transform, a per-mode tridiagonal solve in z and
// the backward transform.  The turn nodes are Dirichlet nodes of the CG
// system, so the preconditioner is applied to the residual (zero there) and
// its result projected onto the free nodes (a principal block of a symmetric
// positive definite inverse).
//
// Layout: one cluster of up to 16 CTAs.  CTA c owns a band of interior rows
// (residual, vectors, stencil, transforms) and the modes m = c, c + C, ...
// (tridiagonal solves).  The radial eigenbasis V sits in shared memory (one
// copy, float4 quads XOR-swizzled so that both transforms read it without
// bank conflicts) when it fits.  The two transposes of an iteration (band
// rows -> modes, modes -> band rows plus one halo row on each side) are
// stores into the owners' shared memory through the cluster's distributed
// shared memory.  The per-mode z systems are solved by one warp each with the
// partition method: every lane eliminates the interior rows of its chunk,
// the chunks' last rows form a reduced tridiagonal system solved by cyclic
// reduction over the lanes with shuffles, and the interior rows follow.  All
// factors of the z systems depend only on chibar and are formed once per
// solve.  Phases are separated by an all-to-all flag barrier in distributed
// shared memory that also carries each CTA's partial sums (release stores,
// acquire loads, every wait bounded: on expiry the barrier records
// PP_ST_TIMEOUT and the kernel runs to its end without further waiting).
// The inner CG is the Chronopoulos-Gear form (both dot products of an
// iteration in one reduction), three barriers per iteration.  FP64 work (a
// small fraction of the FP32 rate on this part) is kept to the refinement
// residual.
#include "pp_internal.h"

#include <cooperative_groups.h>
#include <string>
#include <vector>

namespace cg = cooperative_groups;

namespace pp {

namespace {

constexpr int kCT = 512;                  // threads per CTA
constexpr int kWarps = kCT / 32;
constexpr int kMaxC = 16;                 // CTAs of the cluster
constexpr int kMaxBand = 32;              // interior rows per CTA
constexpr int kLc = 12;                   // z rows per lane of a mode's warp (rows <= 32 kLc)
constexpr int kMaxOuter = 6;              // FP64 refinement steps
constexpr int kMaxInner = 60;             // CG iterations per refinement step
constexpr float kInnerTol = 1e-6f;        // inner residual reduction per refinement step at most (FP32)
constexpr int kPcrLevels = 5;             // cyclic reduction over the 32 lanes
constexpr int kRQ = 3;                    // row quads per warp task of the transforms from global memory

// per-lane factors of the z systems: 5 per interior row (a, 1/pivot,
// c/pivot, responses to the lower and the upper separator), then the
// separator row's two couplings, the reduced system's level multipliers and
// its final reciprocal
constexpr int kFacRow = 5;
constexpr int kFacSep = 2 + 2 * kPcrLevels + 1;

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
    int NR, M, rows;
    double inv2pieps0;
    const float* V;         // radial eigenbasis, M x M row-major ([node][mode])
    const float* VT;        // its transpose ([mode][node]) when V is read from global memory
    const float* zlo;       // per interior row: eps_{i-1} / dz (z coupling below)
    const float* zup;       // eps_i / dz (above)
    const float* zeb;       // (dz / dR) (eps_{i-1} + eps_i) / 2 (radial weight)
    const float* mu;        // radial eigenvalues
    float* chib;            // chibar per node row
    const double* coef0;    // chi-free face coefficients per unknown (4, FP64, set-up)
    const float* coef0f;    // the same in FP32
    double* coef64;         // this solve's coefficients (Eq. epseff with chi), FP64
    float* gvec;            // the CG vectors and FP32 coefficients when they are not in shared memory
    DevState* dst;
    const double* ext;
    int nt;
    double cs, sn;
    double tol;
    PcgPlan pl;
};

__device__ __forceinline__ double tgt_of(const DevState* st, const double* ext, int k, int nt, double cs,
                                         double sn) {
    if (ext) return ext[k];
    // Eq. dirichlet: phi_k = V_c cos + V_s sin with V = V_c - i V_s, plus the
    // retained harmonics
    double vr = st->x[2 * (1 + nt + k)], vi = st->x[2 * (1 + nt + k) + 1];
    const double v1 = vr * cs + (-vi) * sn;
    return st->nharm > 1 ? v1 + harm_turn_sum(st, k, nt, cs, sn) : v1;
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

// barrier words and payloads in each CTA's shared memory: arrive[r] is the
// last generation CTA r announced here, pay[parity][r][v] its partial values
struct Sync {
    unsigned arrive[kMaxC];
    float pay[2][kMaxC][4];
    float red[4][kWarps];   // per-warp partials of this CTA (up to four values)
    int ok;
};

// Cluster barrier with payload: thread t < C reduces the CTA's nv values
// (max if bit v of mxmask, else sum, over the warps' partials in red[v]),
// stores them into CTA t's pay[gen & 1][rank] and announces the generation
// there, then waits until CTA t has announced this generation (or a later
// one) here.  A CTA can be at most one barrier ahead of any other, so the
// payload buffers alternate by generation.  Waits are bounded.
__device__ __forceinline__ void cbar(Sync* sy, unsigned& gen, int C, int rank, DevState* st, int nv,
                                     unsigned mxmask) {
    __syncthreads();
    gen += 1;
    cg::cluster_group cl = cg::this_cluster();
    const int t = threadIdx.x;
    if (t < C) {
        Sync* r = cl.map_shared_rank(sy, t);
        for (int v = 0; v < nv; ++v) {
            const bool mx = (mxmask >> v) & 1u;
            float s = sy->red[v][0];
            for (int w = 1; w < kWarps; ++w) s = mx ? fmaxf(s, sy->red[v][w]) : s + sy->red[v][w];
            r->pay[gen & 1u][rank][v] = s;
        }
        st_release_cluster(&r->arrive[rank], gen);
        int it = 0;
        while ((int)(ld_acquire_cluster(&sy->arrive[t]) - gen) < 0) {
            if (++it > (1 << 24)) {
                atomicOr(&st->status, (unsigned)PP_ST_TIMEOUT);
                sy->ok = 0;
                break;
            }
        }
    }
    __syncthreads();
}

// the cluster-wide value of payload v of the last barrier (every thread, in
// the same order)
__device__ __forceinline__ float pay_all(const Sync* sy, unsigned gen, int C, int v, bool mx) {
    float s = sy->pay[gen & 1u][0][v];
    for (int r = 1; r < C; ++r) s = mx ? fmaxf(s, sy->pay[gen & 1u][r][v]) : s + sy->pay[gen & 1u][r][v];
    return s;
}

// warp partial of one value into red[v]
__device__ __forceinline__ void warp_partial(Sync* sy, int v, float x, bool mx) {
    for (int o = 16; o > 0; o >>= 1) {
        const float u = __shfl_xor_sync(0xffffffffu, x, o);
        x = mx ? fmaxf(x, u) : x + u;
    }
    if ((threadIdx.x & 31) == 0) sy->red[v][threadIdx.x >> 5] = x;
}

// out(r, n, X W[r][n]) for X (nr x ldx, 16-byte aligned rows) and W[k][n] =
// V[k][n] (forward, TRANS = false) or V[n][k] (backward, TRANS = true).  V has
// rows of nqp float4 quads; in shared memory (VSM) the quad index of row R is
// XOR-ed with (R >> 2) & 7, so that the 8 threads of a quarter warp read 8
// different quads in either direction.  A warp task is one quad of rows and
// a block of 8 column quads; its lanes are 4 k-groups x 8 column quads, each
// lane a 4 x 4 tile over its k-group's quarter of k, and the k-groups' tiles
// are added with shuffles (no shared-memory atomics), after which the lanes
// of k-group g hand row g of the tile to `out`.  M is a multiple of 4.
template <bool TRANS, bool VSM, class Out>
__device__ __forceinline__ void transform(const float* X, int ldx, int nr, const float* V, int nqp, int M,
                                          Out out) {
    const int nq = M / 4, nrc = (nr + 3) / 4, ncb = (nq + 7) / 8;
    const int lane = threadIdx.x & 31, kg = lane >> 3, cl8 = lane & 7;
    const int kq_per = (nq + 3) / 4;
    const int kq0 = kg * kq_per, kq1 = min(nq, kq0 + kq_per);
    const float4* V4 = reinterpret_cast<const float4*>(V);
    const float4* X4 = reinterpret_cast<const float4*>(X);
    const int ldx4 = ldx / 4;
    for (int task = threadIdx.x >> 5; task < nrc * ncb; task += kWarps) {
        const int rc = task / ncb, cq = (task % ncb) * 8 + cl8;
        const bool colok = cq < nq;
        const int cqs = colok ? cq : nq - 1;      // idle lanes read a valid quad
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
        for (int kq = kq0; kq < kq1; ++kq) {
            float4 w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!TRANS) {
                    const int sw = VSM ? (cqs ^ (kq & 7)) : cqs;
                    w[q] = VSM ? V4[(size_t)(4 * kq + q) * nqp + sw] : __ldg(V4 + (size_t)(4 * kq + q) * nqp + sw);
                } else {
                    const int sw = VSM ? (kq ^ (cqs & 7)) : kq;
                    w[q] = VSM ? V4[(size_t)(4 * cqs + q) * nqp + sw] : __ldg(V4 + (size_t)(4 * cqs + q) * nqp + sw);
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = min(rc * 4 + r, nr - 1);
                const float4 x = X4[(size_t)row * ldx4 + kq];
                if (!TRANS) {
                    acc[r][0] = fmaf(x.x, w[0].x, fmaf(x.y, w[1].x, fmaf(x.z, w[2].x, fmaf(x.w, w[3].x, acc[r][0]))));
                    acc[r][1] = fmaf(x.x, w[0].y, fmaf(x.y, w[1].y, fmaf(x.z, w[2].y, fmaf(x.w, w[3].y, acc[r][1]))));
                    acc[r][2] = fmaf(x.x, w[0].z, fmaf(x.y, w[1].z, fmaf(x.z, w[2].z, fmaf(x.w, w[3].z, acc[r][2]))));
                    acc[r][3] = fmaf(x.x, w[0].w, fmaf(x.y, w[1].w, fmaf(x.z, w[2].w, fmaf(x.w, w[3].w, acc[r][3]))));
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        acc[r][c] = fmaf(x.x, w[c].x, fmaf(x.y, w[c].y, fmaf(x.z, w[c].z, fmaf(x.w, w[c].w, acc[r][c]))));
                }
            }
        }
        // the four k-groups' tiles: lanes l, l + 8, l + 16, l + 24
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], 8);
                acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], 16);
            }
        // every lane now holds the full tile; lane group kg hands over row kg
        const int row = rc * 4 + kg;
        if (colok && row < nr) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float v = kg == 0 ? acc[0][c] : kg == 1 ? acc[1][c] : kg == 2 ? acc[2][c] : acc[3][c];
                out(row, 4 * cq + c, v);
            }
        }
    }
}

// The forward-oriented product with W = V read from global memory (V too
// large for shared memory; the backward transform passes the transposed
// copy): the loads of V, not the FMAs, bound it (each quad is an L2 access),
// so a warp task covers RQ row quads of the same 32 columns and every V quad
// loaded serves 4 RQ rows.  Lane layout and reduction as in transform().
template <int RQ, class Out>
__device__ __forceinline__ void transform_g(const float* X, int ldx, int nr, const float* V, int M, Out out) {
    const int nq = M / 4, nrc = (nr + 3) / 4, ncb = (nq + 7) / 8, ngr = (nrc + RQ - 1) / RQ;
    const int lane = threadIdx.x & 31, kg = lane >> 3, cl8 = lane & 7;
    const int kq_per = (nq + 3) / 4;
    const int kq0 = kg * kq_per, kq1 = min(nq, kq0 + kq_per);
    const float4* V4 = reinterpret_cast<const float4*>(V);
    const float4* X4 = reinterpret_cast<const float4*>(X);
    const int ldx4 = ldx / 4;
    for (int task = threadIdx.x >> 5; task < ngr * ncb; task += kWarps) {
        const int rg = task / ncb, cq = (task % ncb) * 8 + cl8;
        const bool colok = cq < nq;
        const int cqs = colok ? cq : nq - 1;      // idle lanes read a valid quad
        float acc[RQ * 4][4];
#pragma unroll
        for (int r = 0; r < RQ * 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
        for (int kq = kq0; kq < kq1; ++kq) {
            float4 w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = __ldg(V4 + (size_t)(4 * kq + q) * nq + cqs);
#pragma unroll
            for (int r = 0; r < RQ * 4; ++r) {
                const int row = min(rg * RQ * 4 + r, nr - 1);
                const float4 x = X4[(size_t)row * ldx4 + kq];
                acc[r][0] = fmaf(x.x, w[0].x, fmaf(x.y, w[1].x, fmaf(x.z, w[2].x, fmaf(x.w, w[3].x, acc[r][0]))));
                acc[r][1] = fmaf(x.x, w[0].y, fmaf(x.y, w[1].y, fmaf(x.z, w[2].y, fmaf(x.w, w[3].y, acc[r][1]))));
                acc[r][2] = fmaf(x.x, w[0].z, fmaf(x.y, w[1].z, fmaf(x.z, w[2].z, fmaf(x.w, w[3].z, acc[r][2]))));
                acc[r][3] = fmaf(x.x, w[0].w, fmaf(x.y, w[1].w, fmaf(x.z, w[2].w, fmaf(x.w, w[3].w, acc[r][3]))));
            }
        }
#pragma unroll
        for (int r = 0; r < RQ * 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], 8);
                acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], 16);
            }
#pragma unroll
        for (int g = 0; g < RQ; ++g) {
            const int row = (rg * RQ + g) * 4 + kg;
            if (colok && row < nr) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float v = kg == 0 ? acc[4 * g][c] : kg == 1 ? acc[4 * g + 1][c]
                                  : kg == 2 ? acc[4 * g + 2][c] : acc[4 * g + 3][c];
                    out(row, 4 * cq + c, v);
                }
            }
        }
    }
}

// first interior row of the band of CTA b
__device__ __forceinline__ int band_lo(int rows, int b, int C) { return rows * b / C; }

// z-system coefficients of interior row i for radial eigenvalue mum: a
// (coupling to row i - 1), b (diagonal), c (coupling to row i + 1), with the
// face factors 1 + (chibar_i + chibar_k) / 2
__device__ __forceinline__ void zcoef(const PcgArgs& a, int i, float mum, float& av, float& bv, float& cv) {
    const float ch = __ldcg(a.chib + i + 1);
    const float flo = 1.f + 0.5f * (ch + __ldcg(a.chib + i));
    const float fup = 1.f + 0.5f * (ch + __ldcg(a.chib + i + 2));
    const float lo = __ldg(a.zlo + i) * flo, up = __ldg(a.zup + i) * fup;
    av = i > 0 ? lo : 0.f;
    cv = i + 1 < a.rows ? up : 0.f;
    bv = fmaf(__ldg(a.zeb + i) * (1.f + ch), mum, -(lo + up));
}

// Factors of a mode's z system for lane `lane` of its warp (fac: the lane's
// first factor, consecutive factors fs floats apart).  The lane's chunk of
// rows [i0, i1) has interior rows i0 .. i1 - 2 and its separator i1 - 1.
// The interior rows are eliminated (Thomas) with the separators below and
// above the chunk as parameters: x_k = y_k + sigma_prev u_k + sigma v_k, u
// and v being the responses to the right-hand sides -a_0 in the first row and
// -c_{n-1} in the last.  The separators satisfy a tridiagonal system
// (A, B, C) whose cyclic reduction over the lanes gives per-level
// multipliers.  Empty chunks are identity rows.  The factors are formed in
// place in shared memory.
__device__ void factor_mode(const PcgArgs& a, int m, int lane, float* fac, int fs) {
    const int Lc = a.pl.Lc, rows = a.rows;
    const int i0 = lane * Lc, i1 = min(i0 + Lc, rows);
    const int n = i1 > i0 ? i1 - i0 - 1 : -1;      // interior rows (-1: empty chunk)
    const float mum = __ldg(a.mu + m);
    float uF = 0.f, vF = 1.f, uL = 1.f, vL = 0.f, as = 0.f, bs = 1.f, cs = 0.f;
    if (n >= 0) {
        float cpp = 0.f, upr = 0.f;                // the previous row's c/pivot and forward u
        for (int k = 0; k < n; ++k) {
            float av, bv, cv;
            zcoef(a, i0 + k, mum, av, bv, cv);
            const float piv = k == 0 ? bv : fmaf(-av, cpp, bv);
            const float ip = 1.f / piv;
            const float cp = cv * ip;
            const float u = (k == 0 ? -av : -av * upr) * ip;
            fac[(kFacRow * k + 0) * fs] = av;
            fac[(kFacRow * k + 1) * fs] = ip;
            fac[(kFacRow * k + 2) * fs] = cp;
            fac[(kFacRow * k + 3) * fs] = u;
            cpp = cp;
            upr = u;
        }
        zcoef(a, i0 + n, mum, as, bs, cs);
        if (n > 0) {
            float un = upr, vn = -cpp;             // row n - 1
            fac[(kFacRow * (n - 1) + 4) * fs] = vn;
            uL = un;
            vL = vn;
            for (int k = n - 2; k >= 0; --k) {
                const float cp = fac[(kFacRow * k + 2) * fs];
                un = fmaf(-cp, un, fac[(kFacRow * k + 3) * fs]);
                vn = -cp * vn;
                fac[(kFacRow * k + 3) * fs] = un;
                fac[(kFacRow * k + 4) * fs] = vn;
            }
            uF = un;
            vF = vn;
        }
    }
    // the next chunk's first-row responses (its first row is its separator
    // when it has no interior rows)
    const float uFn = __shfl_down_sync(0xffffffffu, uF, 1);
    const float vFn = __shfl_down_sync(0xffffffffu, vF, 1);
    if (lane == 31) cs = 0.f;
    float A = 0.f, B = 1.f, Cc = 0.f;
    if (n >= 0) {
        A = as * uL;
        B = fmaf(cs, uFn, fmaf(as, vL, bs));
        Cc = cs * vFn;
    }
    float* fs0 = fac + kFacRow * (Lc - 1) * fs;    // separator block
    fs0[0] = as;
    fs0[fs] = cs;
#pragma unroll
    for (int l = 0; l < kPcrLevels; ++l) {
        const int st = 1 << l;
        const float Am = __shfl_up_sync(0xffffffffu, A, st), Bm = __shfl_up_sync(0xffffffffu, B, st);
        const float Cm = __shfl_up_sync(0xffffffffu, Cc, st);
        const float Ap = __shfl_down_sync(0xffffffffu, A, st), Bp = __shfl_down_sync(0xffffffffu, B, st);
        const float Cp = __shfl_down_sync(0xffffffffu, Cc, st);
        const float al = lane >= st ? -A / Bm : 0.f;
        const float ga = lane + st < 32 ? -Cc / Bp : 0.f;
        fs0[(2 + 2 * l) * fs] = al;
        fs0[(3 + 2 * l) * fs] = ga;
        const float A2 = al * Am, C2 = ga * Cp;
        B = fmaf(ga, Ap, fmaf(al, Cm, B));
        A = A2;
        Cc = C2;
    }
    fs0[(2 + 2 * kPcrLevels) * fs] = 1.f / B;
}

// One mode's z solve with the factors, in place on the lane's chunk dd of
// right-hand sides (interior rows, then the separator).
__device__ __forceinline__ void solve_mode(const PcgArgs& a, int lane, const float* fac, int fs, float* dd) {
    const int Lc = a.pl.Lc, rows = a.rows;
    const int i0 = lane * Lc, i1 = min(i0 + Lc, rows);
    const int n = i1 > i0 ? i1 - i0 - 1 : -1;
    float yF = 0.f, yL = 0.f, dsep = 0.f;
    if (n > 0) {
        float prev = 0.f;
        for (int k = 0; k < n; ++k) {
            const float dk = k == 0 ? dd[0] : fmaf(-fac[(kFacRow * k + 0) * fs], prev, dd[k]);
            prev = dk * fac[(kFacRow * k + 1) * fs];
            dd[k] = prev;
        }
        yL = prev;
        float nx = prev;
        for (int k = n - 2; k >= 0; --k) {
            nx = fmaf(-fac[(kFacRow * k + 2) * fs], nx, dd[k]);
            dd[k] = nx;
        }
        yF = nx;
    }
    if (n >= 0) dsep = dd[n];
    const float yFn = __shfl_down_sync(0xffffffffu, yF, 1);
    const float* fs0 = fac + kFacRow * (Lc - 1) * fs;
    float D = n >= 0 ? fmaf(-fs0[0], yL, fmaf(-fs0[fs], yFn, dsep)) : 0.f;
#pragma unroll
    for (int l = 0; l < kPcrLevels; ++l) {
        const int st = 1 << l;
        const float Dm = __shfl_up_sync(0xffffffffu, D, st);
        const float Dp = __shfl_down_sync(0xffffffffu, D, st);
        D = fmaf(fs0[(3 + 2 * l) * fs], Dp, fmaf(fs0[(2 + 2 * l) * fs], Dm, D));
    }
    const float sig = D * fs0[(2 + 2 * kPcrLevels) * fs];
    float sigp = __shfl_up_sync(0xffffffffu, sig, 1);
    if (lane == 0) sigp = 0.f;
    for (int k = 0; k < n; ++k)
        dd[k] = fmaf(sig, fac[(kFacRow * k + 4) * fs], fmaf(sigp, fac[(kFacRow * k + 3) * fs], dd[k]));
    if (n >= 0) dd[n] = sig;
}

}  // namespace

template <bool VSM>
__global__ void __launch_bounds__(kCT, 1) pcg_cluster(PcgArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Sync sy;
    __shared__ int s_band[kMaxC + 1];       // first interior row of each band
    __shared__ int s_rowdst[32 * kLc];      // per interior row: band, local row, halo flags

    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int C = (int)cl.num_blocks();
    const PcgPlan& pl = a.pl;
    const int M = a.M, NR = a.NR, rows = a.rows, Mp = pl.Mp;
    const int lo = band_lo(rows, rank, C), hi = band_lo(rows, rank + 1, C);
    const int nb = hi - lo, nbM = nb * M;
    const int nqp = VSM ? Mp / 4 : M / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nm = (M - rank + C - 1) / C;               // modes of this CTA
    const int fs = pl.nm_max * 32;                       // factor stride (floats)

    const float* Vs = VSM ? reinterpret_cast<const float*>(smem + pl.off_V) : a.V;
    float* s_in = reinterpret_cast<float*>(smem + pl.off_in);      // (nbmax + 2) x Mp, backward input
    float* s_d = reinterpret_cast<float*>(smem + pl.off_d);        // nm_max x rows, z right-hand sides
    unsigned char* s_free = smem + pl.off_free;                    // (nbmax + 2) x M
    float* s_fac = reinterpret_cast<float*>(smem + pl.off_fac);
    double* s_chi = reinterpret_cast<double*>(smem + pl.off_chi);  // set-up only (may share the exchange and factor buffers)
    float *R, *DX, *P, *S, *W, *ZF, *CF;
    {
        const size_t bM = (size_t)pl.nbmax * M;
        float* vb = pl.vec_sm ? reinterpret_cast<float*>(smem + pl.off_vec) : a.gvec + (size_t)rank * pl.gvec_stride;
        R = vb;
        DX = vb + bM;
        P = vb + 2 * bM;
        S = vb + 3 * bM;
        W = vb + 4 * bM;
        ZF = vb + 5 * bM;                  // (nbmax + 2) x M: z with one halo row on each side
        CF = ZF + bM + 2 * (size_t)M;      // 4 per band unknown
    }
    if (threadIdx.x < kMaxC) sy.arrive[threadIdx.x] = 0u;
    if (threadIdx.x == 0) sy.ok = 1;
    unsigned gen = 0;

    // the eigenbasis into shared memory (swizzled quads)
    if (VSM) {
        float4* V4s = reinterpret_cast<float4*>(smem + pl.off_V);
        const float4* V4g = reinterpret_cast<const float4*>(a.V);
        const int nq = M / 4;
        for (int q = threadIdx.x; q < M * nq; q += kCT) {
            const int R0 = q / nq, Q = q % nq;
            V4s[(size_t)R0 * nqp + (Q ^ ((R0 >> 2) & 7))] = __ldg(V4g + q);
        }
    }
    for (int b = threadIdx.x; b <= C; b += kCT) s_band[b] = band_lo(rows, b, C);
    __syncthreads();
    // where each interior row goes after the z solves: its band (local row
    // i - lo + 1), and the upper halo row of the band below it or the lower
    // halo row of the band above it
    for (int i = threadIdx.x; i < rows; i += kCT) {
        int b = i * C / rows;
        while (b + 1 < C && s_band[b + 1] <= i) ++b;
        while (b > 0 && s_band[b] > i) --b;
        int e = (i - s_band[b] + 1) | (b << 8);
        if (i == s_band[b] && b > 0) e |= 1 << 16;
        if (i == s_band[b + 1] - 1 && b + 1 < C) e |= 1 << 17;
        s_rowdst[i] = e;
    }
    cl.sync();                                     // every CTA's barrier words initialised

    // node rows lo .. hi + 1 (the band's interior rows and one halo row on
    // each side) are contiguous in the node grid
    const int hn = (nb + 2) * NR;
    const size_t n0 = (size_t)lo * NR;
    for (int q = threadIdx.x; q < hn; q += kCT) s_chi[q] = node_chi(a, (int)(n0 + q));
    for (int q = threadIdx.x; q < (nb + 2) * M; q += kCT) {
        const int rr = q / M, j = q % M, gi = lo - 1 + rr;
        s_free[q] = (gi >= 0 && gi < rows && a.turn_mask[(gi + 1) * NR + j] < 0) ? 1 : 0;
    }
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
            if (!s_free[li + M]) continue;
            const size_t n = (size_t)(lo + li / M + 1) * NR + li % M;
            const double pc = a.phi[n];
            if (have) a.phi[n] = 2.0 * pc - a.phi_prev[n];
            a.phi_prev[n] = pc;
        }
    }
    cbar(&sy, gen, C, rank, a.dst, 0, 0u);

    float scale = 0.f, rel_last = 0.f;
    bool conv = false, factored = false;
    int inner_total = 0, outer = 0;
    const float tolf = (float)a.tol;
    for (;; ++outer) {
        // ---- FP64 residual r = b - A phi on the band (payload 0: max |r|,
        // 1: the componentwise scale of the first pass); the face coefficients
        // are the set-up's chi-free ones times the factor of Eq. epseff
        float rmax = 0.f, smax = 0.f;
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
            if (!s_free[li + M]) {
                const double diag = c0 + c1 + c2 + c3;
                const double tg = tgt_of(a.dst, a.ext, a.turn_mask[n], a.nt, a.cs, a.sn);
                rmax = fmaxf(rmax, (float)(fabs(tg - pc) * diag));
                if (outer == 0) smax = fmaxf(smax, (float)(fabs(tg) * diag));
            } else {
                const double pu = a.phi[n + NR], pd = a.phi[n - NR], pr = a.phi[n + 1];
                const double pl_ = j > 0 ? a.phi[n - 1] : pc;
                const double qe = a.rho64_e ? a.rho64_e[n] : (double)a.rho_e[n];
                const double qi = a.rho64_e ? a.rho64_i[n] : (double)a.rho_i[n];
                const double b = -((qe + qi) + a.win[n]) * a.inv2pieps0;
                // b - sum_f c_f (phi_f - phi_c) in fused form
                const double ap = fma(c3, pl_ - pc, fma(c2, pr - pc, fma(c1, pd - pc, c0 * (pu - pc))));
                const double r = b - ap;
                rmax = fmaxf(rmax, (float)fabs(r));
                if (outer == 0)
                    smax = fmaxf(smax, (float)(fabs(b) + fabs(c0 * (pu - pc)) + fabs(c1 * (pd - pc)) +
                                              fabs(c2 * (pr - pc)) + fabs(c3 * (pl_ - pc))));
                // inner system B dx = -r with B = -A (positive definite)
                rv = (float)(-r);
            }
            R[li] = rv;
            DX[li] = 0.f;
        }
        warp_partial(&sy, 0, rmax, true);
        warp_partial(&sy, 1, smax, true);
        cbar(&sy, gen, C, rank, a.dst, 2, 3u);
        if (outer == 0) scale = pay_all(&sy, gen, C, 1, true);
        const float rabs = pay_all(&sy, gen, C, 0, true);
        rel_last = scale > 0.f ? rabs / scale : 0.f;
        conv = rabs <= tolf * scale;
        if (conv || outer == kMaxOuter || !sy.ok) break;

        // ---- once per solve (chibar is fixed for the solve): the z factors;
        // the backward input's rows outside the interior are zero (the
        // set-up's chi rows may have used the same memory)
        if (!factored) {
            for (int q = threadIdx.x; q < (pl.nbmax + 2) * Mp; q += kCT) s_in[q] = 0.f;
            for (int lm = warp; lm < nm; lm += kWarps) factor_mode(a, rank + lm * C, lane, s_fac + lm * 32 + lane, fs);
            factored = true;
        }

        // ---- inner CG (Chronopoulos-Gear) on B dx = rho with the projected
        // chibar preconditioner z = -(Pi P_chibar Pi rho)
        float gam = 0.f, alpha = 0.f, thr = 0.f, be = 0.f;
        for (int it = 0;; ++it) {
            // (A) with the scalars of the previous iteration: the new
            // directions p = z + beta p, s = w + beta s, then x += alpha p,
            // rho -= alpha s and max |rho|; the forward transform of rho,
            // each mode's rows stored into its owner's shared memory
            float rmf = 0.f;
            for (int li = threadIdx.x; li < nbM; li += kCT) {
                float rv = R[li];
                if (it > 0 && s_free[li + M]) {
                    const float pv = it == 1 ? ZF[li + M] : fmaf(be, P[li], ZF[li + M]);
                    const float sv = it == 1 ? W[li] : fmaf(be, S[li], W[li]);
                    P[li] = pv;
                    S[li] = sv;
                    DX[li] = fmaf(alpha, pv, DX[li]);
                    rv = fmaf(-alpha, sv, rv);
                    R[li] = rv;
                }
                rmf = fmaxf(rmf, fabsf(rv));
            }
            warp_partial(&sy, 0, rmf, true);
            __syncthreads();
            if constexpr (VSM) {
                transform<false, VSM>(R, M, nb, Vs, nqp, M, [&](int r, int m, float v) {
                    cl.map_shared_rank(s_d, m % C)[(m / C) * rows + lo + r] = v;
                });
            } else {
                transform_g<kRQ>(R, M, nb, a.V, M, [&](int r, int m, float v) {
                    cl.map_shared_rank(s_d, m % C)[(m / C) * rows + lo + r] = v;
                });
            }
            cbar(&sy, gen, C, rank, a.dst, 1, 1u);
            const float rn = pay_all(&sy, gen, C, 0, true);
            // the inner solve stops at half the refinement's target residual
            // (in absolute terms, so that a good initial guess saves
            // iterations), or at the reduction FP32 can deliver
            if (it == 0) thr = fmaxf(0.5f * tolf * scale, kInnerTol * rn);
            if (!sy.ok || rn <= thr || it == kMaxInner) break;
            // (B) z solves of this CTA's modes; each row to the band that holds
            // it (and to the neighbouring band whose halo it is)
            for (int lm = warp; lm < nm; lm += kWarps) {
                const int m = rank + lm * C;
                const int i0 = lane * pl.Lc, i1 = min(i0 + pl.Lc, rows);
                float* dd = s_d + lm * rows + i0;
                solve_mode(a, lane, s_fac + lm * 32 + lane, fs, dd);
                for (int i = i0; i < i1; ++i) {
                    const float x = dd[i - i0];
                    const int e = s_rowdst[i];
                    const int b = (e >> 8) & 0xff, rr = e & 0xff;
                    cl.map_shared_rank(s_in, b)[rr * Mp + m] = x;
                    if (e & (1 << 16))
                        cl.map_shared_rank(s_in, b - 1)[(s_band[b] - s_band[b - 1] + 1) * Mp + m] = x;
                    if (e & (1 << 17)) cl.map_shared_rank(s_in, b + 1)[m] = x;
                }
            }
            cbar(&sy, gen, C, rank, a.dst, 0, 0u);
            // (C) backward transform of the band and its halo rows, projected
            // onto the free nodes: z = -(P rho); w = B z on the band,
            // gamma = rho . z, delta = z . w
            // from global memory the transposed copy is read row-wise, as
            // the forward transform reads V (coalesced quads)
            if constexpr (VSM) {
                transform<true, VSM>(s_in, Mp, nb + 2, Vs, nqp, M, [&](int r, int j, float v) {
                    const int q = r * M + j;
                    ZF[q] = s_free[q] ? -v : 0.f;
                });
            } else {
                transform_g<kRQ>(s_in, Mp, nb + 2, a.VT, M, [&](int r, int j, float v) {
                    const int q = r * M + j;
                    ZF[q] = s_free[q] ? -v : 0.f;
                });
            }
            __syncthreads();
            float pgf = 0.f, pdf = 0.f;
            for (int li = threadIdx.x; li < nbM; li += kCT) {
                float wv = 0.f;
                const int q = li + M;
                const float zc = ZF[q];
                if (s_free[q]) {
                    const int j = li % M;
                    const float* c = CF + 4 * li;
                    const float zr = j + 1 < M ? ZF[q + 1] : 0.f;
                    float y = c[0] * (ZF[q + M] - zc) + c[1] * (ZF[q - M] - zc) + c[2] * (zr - zc);
                    if (j > 0) y += c[3] * (ZF[q - 1] - zc);
                    wv = -y;
                }
                W[li] = wv;
                pgf = fmaf(R[li], zc, pgf);
                pdf = fmaf(zc, wv, pdf);
            }
            warp_partial(&sy, 0, pgf, false);
            warp_partial(&sy, 1, pdf, false);
            cbar(&sy, gen, C, rank, a.dst, 2, 0u);
            // (D) the scalars (every thread, in the same order) and the new
            // directions
            const float gn = pay_all(&sy, gen, C, 0, false), dn = pay_all(&sy, gen, C, 1, false);
            float al;
            if (it == 0) {
                be = 0.f;
                al = dn > 0.f ? gn / dn : 0.f;
            } else {
                be = gam != 0.f ? gn / gam : 0.f;
                const float den = dn - be * gn / alpha;
                al = den > 0.f ? gn / den : 0.f;
            }
            alpha = al;
            gam = gn;
            ++inner_total;
        }
        // phi += dx on the free nodes of the band; the next residual reads the
        // neighbours' rows after the barrier
        for (int li = threadIdx.x; li < nbM; li += kCT)
            if (s_free[li + M]) a.phi[(size_t)(lo + li / M + 1) * NR + li % M] += (double)DX[li];
        cbar(&sy, gen, C, rank, a.dst, 0, 0u);
        if (!sy.ok) break;
    }
    if (rank == 0 && threadIdx.x == 0) {
        DevState* st = a.dst;
        st->prel = (double)rel_last;
        st->piters = inner_total + outer;
        st->pdone = 1;
        if (a.extrapolate) st->phi_prev_ok = 1;
        if (!conv) st->status |= PP_ST_NOCONV;
    }
    cl.sync();                                     // no CTA leaves while others may write its shared memory
}

// ---------------------------------------------------------------- host side
namespace {
constexpr size_t kSmemMax = 224 * 1024;   // dynamic shared memory of one CTA (the barrier and row tables are static)

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// The shared-memory plan for a cluster of C CTAs: the exchange buffers, the
// free-node mask and the z factors always; the band vectors, and then V, when
// they fit.
bool plan_for(const Cell* c, int C, PcgPlan& p) {
    const int M = c->ps.M, rows = c->ps.rows, NR = c->NR;
    p.C = C;
    p.nbmax = (rows + C - 1) / C;
    p.Mp = (M + 31) & ~31;
    p.nm_max = (M + C - 1) / C;
    p.Lc = (rows + 31) / 32;
    if (p.nbmax > kMaxBand || p.nm_max > kWarps || p.Lc > kLc || rows < C) return false;
    const size_t fac = sizeof(float) * (size_t)(kFacRow * (p.Lc - 1) + kFacSep) * p.nm_max * 32;
    const size_t sin_ = sizeof(float) * (size_t)(p.nbmax + 2) * p.Mp;
    const size_t sd = sizeof(float) * (size_t)p.nm_max * rows;
    const size_t sfree = (size_t)(p.nbmax + 2) * M;
    const size_t schi = sizeof(double) * (size_t)(p.nbmax + 2) * NR;
    const size_t vec = sizeof(float) * ((size_t)10 * p.nbmax * M + (size_t)2 * M);
    const size_t vsz = sizeof(float) * (size_t)M * p.Mp;
    // the set-up's chi rows share the exchange buffers and the z factors,
    // which are first written after the last use of chi
    const size_t xch = align16(sin_) + align16(sd) + align16(fac);
    const bool chi_own = schi > xch;
    const size_t base = xch + align16(sfree) + (chi_own ? align16(schi) : 0);
    if (base > kSmemMax) return false;
    p.vec_sm = base + align16(vec) <= kSmemMax ? 1 : 0;
    p.v_sm = p.vec_sm && base + align16(vec) + align16(vsz) <= kSmemMax ? 1 : 0;
    size_t o = 0;
    p.off_V = -1;
    p.off_vec = -1;
    if (p.v_sm) {
        p.off_V = (long long)o;
        o += align16(vsz);
    }
    if (p.vec_sm) {
        p.off_vec = (long long)o;
        o += align16(vec);
    }
    p.off_free = (long long)o;
    o += align16(sfree);
    p.off_in = (long long)o;
    p.off_d = (long long)(o + align16(sin_));
    p.off_fac = (long long)(o + align16(sin_) + align16(sd));
    p.off_chi = (long long)o;
    o += xch;
    if (chi_own) {
        p.off_chi = (long long)o;
        o += align16(schi);
    }
    p.smem = o;
    p.gvec_stride = (long long)(vec / sizeof(float));
    return true;
}

template <bool VSM>
bool cluster_schedulable(int C, size_t shm) {
    // the largest dynamic shared memory any plan uses, so that cells with
    // different plans share the kernel
    if (cudaFuncSetAttribute(pcg_cluster<VSM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(pcg_cluster<VSM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax) !=
            cudaSuccess) {
        cudaGetLastError();
        return false;
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
    if (cudaOccupancyMaxActiveClusters(&n, pcg_cluster<VSM>, &cfg) == cudaSuccess && n > 0) return true;
    cudaGetLastError();
    return false;
}

// 16 CTAs when the device schedules such clusters (non-portable size) with
// the plan's shared memory, else 8
bool choose_plan(const Cell* c, PcgPlan& out) {
    for (int C = 16; C >= 8; C /= 2) {
        PcgPlan p;
        if (!plan_for(c, C, p)) continue;
        const bool ok = p.v_sm ? cluster_schedulable<true>(C, p.smem) : cluster_schedulable<false>(C, p.smem);
        if (ok) {
            out = p;
            return true;
        }
    }
    return false;
}
}  // namespace

int pcg_supported(Cell* c) {
    const int M = c->ps.M;
    if (!(M % 4 == 0 && M >= 8)) return 0;
    PcgPlan p;
    if (!choose_plan(c, p)) return 0;
    c->pcg_plan = p;
    c->pcg_blocks = p.C;
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
    const PcgPlan& p = c->pcg_plan;
    // private per-CTA global regions for the band vectors when they are not in
    // shared memory
    c->d_pcg32 = p.vec_sm ? nullptr : c->alloc<float>((size_t)p.C * p.gvec_stride);
    if (!p.v_sm) {
        // the transposed eigenbasis for the backward transform from global memory
        std::vector<float> v((size_t)M * M), vt((size_t)M * M);
        cudaMemcpy(v.data(), c->ps.Vf, sizeof(float) * v.size(), cudaMemcpyDeviceToHost);
        for (int r = 0; r < M; ++r)
            for (int q = 0; q < M; ++q) vt[(size_t)q * M + r] = v[(size_t)r * M + q];
        c->d_pcg_VT = c->alloc<float>(vt.size());
        cudaMemcpy(c->d_pcg_VT, vt.data(), sizeof(float) * vt.size(), cudaMemcpyHostToDevice);
    }
    c->d_pcg_chib = c->alloc<float>((size_t)c->NZ + 2);
    c->d_phi_prev = c->alloc<double>(c->nnodes);
}

int pcg_refine(Cell* c, double cs, double sn, cudaStream_t st, const double* ext, bool in_step) {
    const PcgPlan& p = c->pcg_plan;
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
    a.inv2pieps0 = 1.0 / (2.0 * kPi * kEps0);
    a.V = c->ps.Vf;
    a.VT = c->d_pcg_VT;
    a.zlo = c->d_pcg_zrow;
    a.zup = c->d_pcg_zrow + a.rows;
    a.zeb = c->d_pcg_zrow + 2 * a.rows;
    a.mu = c->d_pcg_mu;
    a.chib = c->d_pcg_chib;
    a.coef0 = c->d_pcg0;
    a.coef0f = c->d_pcg0f;
    a.coef64 = c->d_pcg;
    a.gvec = c->d_pcg32;
    a.dst = c->d_st;
    a.ext = ext;
    a.nt = c->nturns;
    a.cs = cs;
    a.sn = sn;
    a.tol = c->cfg.poisson_tol;
    a.pl = p;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.C);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e =
        p.v_sm ? cudaLaunchKernelEx(&cfg, pcg_cluster<true>, a) : cudaLaunchKernelEx(&cfg, pcg_cluster<false>, a);
    count_launch();
    if (e != cudaSuccess) {
        set_error(std::string("Poisson cluster launch: ") + cudaGetErrorString(e));
        return PP_E_CUDA;
    }
    return 0;
}

}  // namespace pp
