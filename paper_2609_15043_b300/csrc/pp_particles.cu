// Particle kernels: the fused gather / cylindrical Boris push / boundaries /
// null-collision MCC / deposition kernel, the append of ionisation products
// ordered by parent uid, and the counting sort that keeps the store in cell
// order.
//
// Arithmetic of the decision path is plain IEEE float32 with no contraction
// (the library is built with --fmad=false), in the same operation order as the
// float32 instantiation of the oracle, so cell crossings, absorptions and
// collision decisions of a step are reproduced exactly.
#include "pp_internal.h"
#include "pp_mcc.cuh"

#include <climits>

namespace pp {

// ---------------------------------------------------------------- TMA bulk copies
// 1-D bulk copies between global and shared memory (cp.async.bulk), completed
// through an mbarrier transaction count; sizes and addresses are multiples of
// 16 bytes (chunk bases are multiples of the chunk size; storage is padded).
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// bounded wait: false when the phase did not complete within the limit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    uint32_t addr = smem_u32(bar);
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------- deposition
// Register accumulator of the bilinear node weights of one cell.  A thread's
// particles are consecutive in the cell-sorted store, so most of them share
// the accumulated cell.
struct DepAcc {
    int iz, ir;       // accumulated cell; iz = -1 when empty
    float v0, v1, v2, v3;
};

struct Tile {
    float* s;      // shared nodes: rows [lo, lo + rows) x columns [clo, clo + cols), row stride cols
    int lo, rows;
    int clo, cols;
    float* g;      // global node grid
    int NR;
};

// shared and global targets take separate branches so that each compiles to
// the native atomic of its state space (a pointer that may be either would
// force generic atomics)
__device__ __forceinline__ void tile_add4(const Tile& t, int iz, int ir, float v0, float v1, float v2, float v3) {
    const int r0 = iz - t.lo, c0 = ir - t.clo;
    // both corner rows and both corner columns inside the tile
    if (r0 >= 0 && r0 + 1 < t.rows && c0 >= 0 && c0 + 1 < t.cols) {
        uint32_t a = smem_u32(t.s + r0 * t.cols + c0);
        uint32_t b = a + 4u * (uint32_t)t.cols;
        asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v0));
        asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a + 4u), "f"(v1));
        asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(b), "f"(v2));
        asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(b + 4u), "f"(v3));
    } else {
        float* p = t.g + iz * t.NR + ir;
        atomicAdd(p, v0);
        atomicAdd(p + 1, v1);
        atomicAdd(p + t.NR, v2);
        atomicAdd(p + t.NR + 1, v3);
    }
}

// current deposit: the run of sorted old cells only moves forward, so a new
// cell flushes the previous one
__device__ __forceinline__ void dep_run(DepAcc& a, const Tile& t, int iz, int ir, float v0, float v1, float v2,
                                        float v3) {
    if (iz != a.iz || ir != a.ir) {
        if (a.iz >= 0) tile_add4(t, a.iz, a.ir, a.v0, a.v1, a.v2, a.v3);
        a.iz = iz;
        a.ir = ir;
        a.v0 = v0;
        a.v1 = v1;
        a.v2 = v2;
        a.v3 = v3;
    } else {
        a.v0 += v0;
        a.v1 += v1;
        a.v2 += v2;
        a.v3 += v3;
    }
}

// charge deposit at the new positions: slot a holds the first cell (the
// "home" cell most particles stay in), slot b the last other cell, so strays
// that land in the same neighbour accumulate too; a third cell evicts b
__device__ __forceinline__ void dep_home(DepAcc& a, DepAcc& b, const Tile& t, int iz, int ir, float v0, float v1,
                                         float v2, float v3) {
    if (iz == a.iz && ir == a.ir) {
        a.v0 += v0;
        a.v1 += v1;
        a.v2 += v2;
        a.v3 += v3;
    } else if (iz == b.iz && ir == b.ir) {
        b.v0 += v0;
        b.v1 += v1;
        b.v2 += v2;
        b.v3 += v3;
    } else if (a.iz < 0) {
        a.iz = iz;
        a.ir = ir;
        a.v0 = v0;
        a.v1 = v1;
        a.v2 = v2;
        a.v3 = v3;
    } else {
        if (b.iz >= 0) tile_add4(t, b.iz, b.ir, b.v0, b.v1, b.v2, b.v3);
        b.iz = iz;
        b.ir = ir;
        b.v0 = v0;
        b.v1 = v1;
        b.v2 = v2;
        b.v3 = v3;
    }
}

// End-of-chunk flush: segmented inclusive scan over the warp's lanes (lanes
// hold consecutive particle runs, so equal cells sit in adjacent lanes); the
// last lane of every segment adds the segment's sums.  All lanes call it.
__device__ __forceinline__ void dep_flush_warp(DepAcc& a, const Tile& t) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int key = (a.iz >= 0) ? a.iz * t.NR + a.ir : -1;
    int kl = __shfl_up_sync(full, key, 1);
    unsigned f = (lane == 0 || kl != key) ? 1u : 0u;    // segment head
    const unsigned head = f;
    float s0 = a.v0, s1 = a.v1, s2 = a.v2, s3 = a.v3;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float u0 = __shfl_up_sync(full, s0, o);
        float u1 = __shfl_up_sync(full, s1, o);
        float u2 = __shfl_up_sync(full, s2, o);
        float u3 = __shfl_up_sync(full, s3, o);
        unsigned fu = __shfl_up_sync(full, f, o);
        if (lane >= o) {
            if (!f) {
                s0 += u0;
                s1 += u1;
                s2 += u2;
                s3 += u3;
            }
            f |= fu;
        }
    }
    unsigned next_head = __shfl_down_sync(full, head, 1);
    bool tail = (lane == 31) || next_head;
    if (tail && key >= 0) tile_add4(t, a.iz, a.ir, s0, s1, s2, s3);
    a.iz = -1;
}

// ---------------------------------------------------------------- push kernel
struct PushArgs {
    ParticleBuf p[2];
    const int* nslot;
    SpeciesConst sp[2];
    const float* F;
    float* rho[2];                  // per species (the susceptibility needs them apart)
    float* jm;
    double* win;
    int nr, NR, i_win;
    int implicit;                   // direct-implicit electrostatics
    uint32_t div_magic, div_shift;  // cell / nr = umulhi(cell, magic) >> shift
    const unsigned long long* step;  // device step counter (RNG counter word)
    uint32_t key0, key1;
    Event* ev;
    int ev_cap;
    DevState* st;
};

static_assert(kTileRows <= kPushThreads / 32, "one warp clears and flushes each tile row");

// shared-memory layout of one block (dynamic)
struct PushSmem {
    static constexpr int kArrays = 7;        // cell, dr, dz, vr, vt, vz, uid
    static size_t bytes(int NR, int ppt) {
        const size_t ch = (size_t)kPushThreads * ppt;
        return sizeof(float) * ch * kArrays + sizeof(float) * 2 * kTileRows * NR + sizeof(uint16_t) * ch + 256;
    }
};

// One block owns a chunk of 256 PPT consecutive particles of one species at a
// time: TMA bulk copies bring the seven SoA slices into shared memory, each
// thread advances PPT consecutive particles (gather, Boris, current and
// charge deposits accumulated in registers, move, boundaries, null test), the
// few collision candidates are then processed densely, and bulk copies write
// the six updated slices back.  W: per-particle relative weights, read
// through the read-only cache (each thread's PPT consecutive weights share
// cache lines; staging them would cost the shared memory of the third block
// per SM); each particle's charge is then (q W_s) w.  Ions absorbed on a
// surface may emit a secondary electron (see_emit).
// PPT (particles per thread, a power of two up to 16) sets the chunk, the
// tile shape the autotuner chooses; IMPL selects the direct-implicit form at
// compile time.
template <bool W, int PPT, bool IMPL>
__global__ void __launch_bounds__(kPushThreads, PP_PUSH_MINB) push_kernel(PushArgs a) {
    constexpr int kCh = kPushThreads * PPT;
    static_assert(PPT >= 1 && PPT <= kPptMax && (PPT & (PPT - 1)) == 0, "PPT: a power of two up to kPptMax");
    extern __shared__ __align__(128) unsigned char smem[];
    uint32_t* s_cell = reinterpret_cast<uint32_t*>(smem);
    float* s_dr = reinterpret_cast<float*>(s_cell + kCh);
    float* s_dz = s_dr + kCh;
    float* s_vr = s_dz + kCh;
    float* s_vt = s_vr + kCh;
    float* s_vz = s_vt + kCh;
    uint32_t* s_uid = reinterpret_cast<uint32_t*>(s_vz + kCh);
    float* t_rho = reinterpret_cast<float*>(s_uid + kCh);
    float* t_jm = t_rho + kTileRows * a.NR;
    uint16_t* s_cand = reinterpret_cast<uint16_t*>(t_jm + kTileRows * a.NR);
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_min[kPushThreads / 32], s_max[kPushThreads / 32];
    __shared__ int s_cmin[kPushThreads / 32], s_cmax[kPushThreads / 32];
    __shared__ int s_ncand;
    __shared__ int s_ok;
    __shared__ float s_f[kPushThreads / 32][2];
    __shared__ unsigned s_c[kPushThreads / 32][3];
    __shared__ unsigned s_pc[6];            // collision-pass tallies of the block

    const int n0 = a.nslot[0], n1 = a.nslot[1];
    const int ce = (n0 + kCh - 1) / kCh, ci = (n1 + kCh - 1) / kCh;
    const int nr = a.nr, NR = a.NR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = threadIdx.x;
    const uint32_t step = (uint32_t)(*a.step);
    const CollCtx<float> cc{a.key0, a.key1, a.ev, a.ev_cap, a.st, a.sp[1].vth_gas};

    if (t == 0) {
        mbar_init(&s_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (t < 6) s_pc[t] = 0u;
    __syncthreads();

    float acc_ind = 0.f, acc_es = 0.f;
    // per-thread counters of the push: 0 pushed, 1 absorbed e, 2 absorbed i
    // (the collision pass tallies into s_pc: 0 el/cx... see below)
    unsigned cnt[3] = {0, 0, 0};
    uint32_t parity = 0;

    // dynamic schedule: a block takes the next unprocessed chunk when it is
    // done with its last (electron chunks first), which evens out the blocks'
    // shares of cheap and expensive chunks; the next index is taken before the
    // barrier that ends a chunk.  The node tiles start zeroed and every flush
    // zeroes the entries it reads, so a chunk finds its tile clear.
    __shared__ int s_chunk;
    for (int q = t; q < 2 * kTileRows * NR; q += kPushThreads) t_rho[q] = 0.f;   // t_jm follows t_rho
    if (t == 0) s_chunk = atomicAdd(&a.st->push_chunk, 1);
    __syncthreads();
    for (;;) {
        const int chunk = s_chunk;
        if (chunk >= ce + ci) break;
        const int sp = chunk < ce ? 0 : 1;
        const int base = (chunk - (sp ? ce : 0)) * kCh;
        const int n = sp ? n1 : n0;
        const int nact = min(kCh, n - base);
        const ParticleBuf P = a.p[sp];
        const SpeciesConst S = a.sp[sp];
        const uint32_t bytes = (uint32_t)((nact * 4 + 15) & ~15);

        // ---- stage the chunk (previous bulk stores must have read their smem)
        if (t == 0) {
            bulk_wait_read();
            mbar_expect_tx(&s_bar, 7u * bytes);
            bulk_g2s(s_cell, P.cell + base, bytes, &s_bar);
            bulk_g2s(s_dr, P.dr + base, bytes, &s_bar);
            bulk_g2s(s_dz, P.dz + base, bytes, &s_bar);
            bulk_g2s(s_vr, P.vr + base, bytes, &s_bar);
            bulk_g2s(s_vt, P.vt + base, bytes, &s_bar);
            bulk_g2s(s_vz, P.vz + base, bytes, &s_bar);
            bulk_g2s(s_uid, P.uid + base, bytes, &s_bar);
            s_ncand = 0;
        }
        bool ok = mbar_wait(&s_bar, parity);
        if (!ok) {
            atomicOr(&a.st->status, (unsigned)PP_ST_TIMEOUT);
            mbar_wait(&s_bar, parity);        // give the copies in flight a second bounded wait
        }
        parity ^= 1u;
        if (t == 0) s_ok = ok ? 1 : 0;
        // ---- node tile from the chunk's cell rows and columns: deposits at the
        // old positions reach one row/column beyond, at the new ones one
        // below and two beyond; anything outside goes to global atomics
        int lmin = INT_MAX, lmax = -1, cmin = INT_MAX, cmax = -1;
        for (int q = t; q < nact; q += kPushThreads) {
            uint32_t c = s_cell[q];
            if (c != kDead) {
                int iz = (int)(__umulhi(c, a.div_magic) >> a.div_shift);
                int ir = (int)c - iz * nr;
                lmin = min(lmin, iz);
                lmax = max(lmax, iz);
                cmin = min(cmin, ir);
                cmax = max(cmax, ir);
            }
        }
        lmin = __reduce_min_sync(0xffffffffu, lmin);
        lmax = __reduce_max_sync(0xffffffffu, lmax);
        cmin = __reduce_min_sync(0xffffffffu, cmin);
        cmax = __reduce_max_sync(0xffffffffu, cmax);
        if (lane == 0) {
            s_min[warp] = lmin;
            s_max[warp] = lmax;
            s_cmin[warp] = cmin;
            s_cmax[warp] = cmax;
        }
        __syncthreads();
        if (!s_ok) break;
        int bmin = INT_MAX, bmax = -1, bcmin = INT_MAX, bcmax = -1;
        for (int w = 0; w < kPushThreads / 32; ++w) {
            bmin = min(bmin, s_min[w]);
            bmax = max(bmax, s_max[w]);
            bcmin = min(bcmin, s_cmin[w]);
            bcmax = max(bcmax, s_cmax[w]);
        }
        // the implicit correction moves a particle by less than a cell: the
        // tile then spans one more row and column on each side
        const int pad = IMPL ? 1 : 0;
        const int tlo = max(bmin - 1 - pad, 0);
        const int thi = min(bmax + 2 + pad, a.i_win);
        const int trows = (bmax < 0) ? 0 : min(thi - tlo + 1, kTileRows);
        const int tclo = max(bcmin - 1 - pad, 0);
        const int tcols = (bmax < 0) ? 0 : min(bcmax + 2 + pad, nr) - tclo + 1;
        float* const rho_sp = a.rho[sp];
        const Tile tj{t_jm, tlo, trows, tclo, tcols, a.jm, NR};
        const Tile tq{t_rho, tlo, trows, tclo, tcols, rho_sp, NR};

        // ---- phase A: thread-contiguous push
        DepAcc dj{-1, 0, 0.f, 0.f, 0.f, 0.f};
        DepAcc dq{-1, 0, 0.f, 0.f, 0.f, 0.f};
        DepAcc dq2{-1, 0, 0.f, 0.f, 0.f, 0.f};
        uint32_t fcell = kDead;
        float4 f0, f1, f2, f3, f4;
        // thread t owns particles t*PPT .. t*PPT + PPT-1 and visits them
        // starting at offset t/(32/PPT): the 32 lanes of a warp then hit 32
        // different banks
        const int p0 = t * PPT, rot = (t / (32 / PPT)) & (PPT - 1);
#pragma unroll 1
        for (int k = 0; k < PPT; ++k) {
            const int p = p0 + ((k + rot) & (PPT - 1));
            if (p >= nact) continue;
            const uint32_t cell = s_cell[p];
            if (cell == kDead) continue;
            const int iz0 = (int)(__umulhi(cell, a.div_magic) >> a.div_shift);
            const int ir0 = (int)cell - iz0 * nr;
            const float dr0 = s_dr[p], dz0 = s_dz[p];
            const float vr0 = s_vr[p], vt = s_vt[p], vz0 = s_vz[p];
            const float wrel = W ? __ldg(P.w + base + p) : 1.0f;
            const float wq = W ? S.qw * wrel : S.qw;            // the particle's charge
            // the null-collision uniform depends only on (uid, step, species):
            // drawn first, its integer rounds overlap the floating-point chain
            const uint32_t rnull =
                philox2x32_10(s_uid[p], (step & 0x7FFFFFFFu) | ((uint32_t)sp << 31), a.key0 ^ a.key1);
            if (cell != fcell) {
                const float4* f = reinterpret_cast<const float4*>(a.F) + (size_t)cell * 5;
                f0 = __ldg(f);
                f1 = __ldg(f + 1);
                f2 = __ldg(f + 2);
                f3 = __ldg(f + 3);
                f4 = __ldg(f + 4);
                fcell = cell;
            }
            // gather (bilinear weights at the old position)
            const float one = 1.0f;
            float wa = one - dr0, wb = one - dz0;
            float w00 = wa * wb, w01 = dr0 * wb, w10 = wa * dz0, w11 = dr0 * dz0;
            float Er = w00 * f0.x + w01 * f0.y + w10 * f0.z + w11 * f0.w;
            float Ez = w00 * f1.x + w01 * f1.y + w10 * f1.z + w11 * f1.w;
            float Et = w00 * f2.x + w01 * f2.y + w10 * f2.z + w11 * f2.w;
            float Br = w00 * f3.x + w01 * f3.y + w10 * f3.z + w11 * f3.w;
            float Bz = w00 * f4.x + w01 * f4.y + w10 * f4.z + w11 * f4.w;
            int ir = ir0, iz = iz0;
            float dr = dr0, dz = dz0, vr = vr0, vz = vz0;
            if (IMPL) {
                // the previous step's implicit kick with E^s at the predicted
                // position: v += (q/m) dt E, x += (q/m) dt^2 E (cells), a pass
                // through the axis reflects, leaving the plasma region absorbs
                const float vrc = vr + S.qmd * Er, vzc = vz + S.qmd * Ez;
                float tr = dr + S.kres * Er, tz = dz + S.kzes * Ez;
                float kr = fminf(fmaxf(floorf(tr), -1048576.0f), 1048576.0f);
                tr = tr - kr;
                int irc = ir + (int)kr;
                if (tr >= one) {
                    tr = tr - one;
                    irc += 1;
                }
                float kz = fminf(fmaxf(floorf(tz), -1048576.0f), 1048576.0f);
                tz = tz - kz;
                int izc = iz + (int)kz;
                if (tz >= one) {
                    tz = tz - one;
                    izc += 1;
                }
                float vr_k = vrc;
                if (irc < 0) {
                    const float rpos = -((float)irc + tr);
                    const float jf = floorf(rpos);
                    irc = (int)jf;
                    tr = rpos - jf;
                    vr_k = -vrc;
                }
                const bool ce = izc < 0;
                const bool cw = !ce && irc >= nr;
                const bool cd = !ce && !cw && izc >= a.i_win;
                if (ce || cw || cd) {
                    bool emit = false;
                    if (sp == 1 && S.see_g > 0.0f)
                        emit = see_emit(cc, step, S, s_uid[p], ce ? 0 : (cw ? 1 : 2), cell, dr0, dz0, wrel);
                    if (cd) {
                        const float qd = emit ? wq * 2.0f : wq;
                        float rpos = (float)irc + tr;
                        int j0 = (int)floorf(rpos);
                        float fr = rpos - (float)j0;
                        atomicAdd(&a.win[a.i_win * NR + j0], (double)(qd * (one - fr)));
                        atomicAdd(&a.win[a.i_win * NR + min(j0 + 1, nr)], (double)(qd * fr));
                    }
                    ++cnt[0];
                    ++cnt[1 + sp];
                    s_cell[p] = kDead;
                    s_dr[p] = 0.0f;
                    s_dz[p] = 0.0f;
                    continue;
                }
                // electrostatic work of the kick (mean of the pre- and post-kick velocities)
                acc_es = __fmaf_rn(wq, __fmaf_rn((vr + vrc) * 0.5f, Er, ((vz + vzc) * 0.5f) * Ez), acc_es);
                ir = irc;
                iz = izc;
                dr = tr;
                dz = tz;
                vr = vr_k;
                vz = vzc;
                // the current moment is deposited at the corrected position
                wa = one - dr;
                wb = one - dz;
                w00 = wa * wb;
                w01 = dr * wb;
                w10 = wa * dz;
                w11 = dr * dz;
                Er = 0.0f;      // the Boris step carries E_theta and B only
                Ez = 0.0f;
            }
            // Boris in the local frame (x = r, y = theta, z); B_theta = 0
            float hx = S.qmh * Er, hy = S.qmh * Et, hz = S.qmh * Ez;
            float vmx = vr + hx, vmy = vt + hy, vmz = vz + hz;
            float tx = S.qmh * Br, tz = S.qmh * Bz;
            float t2 = tx * tx + tz * tz;
            float sf = 2.0f / (one + t2);
            float sx = tx * sf, sz = tz * sf;
            float v1x = vmx + vmy * tz;
            float v1y = vmy + (vmz * tx - vmx * tz);
            float v1z = vmz - vmy * tx;
            float vpx = vmx + v1y * sz;
            float vpy = vmy + (v1z * sx - v1x * sz);
            float vpz = vmz - v1y * sx;
            float vnx = vpx + hx, vny = vpy + hy, vnz = vpz + hz;
            // current moment at the old position, time-centred velocity
            float vbt = (vt + vny) * 0.5f;
            float vbr = (vr + vnx) * 0.5f;
            float vbz = (vz + vnz) * 0.5f;
            float jmv = wq * vbt;
            acc_ind = __fmaf_rn(jmv, Et, acc_ind);
            if (!IMPL) acc_es = __fmaf_rn(wq, __fmaf_rn(vbr, Er, vbz * Ez), acc_es);
            ++cnt[0];
            dep_run(dj, tj, iz, ir, jmv * w00, jmv * w01, jmv * w10, jmv * w11);
            // move (cell units): r' = |(r + a, b)| written as r + delta
            float am = vnx * S.dtr, bm = vny * S.dtr, cm = vnz * S.dtz;
            float rho = (float)ir + dr;
            float x1 = rho + am;
            float rp = sqrtf(x1 * x1 + bm * bm);
            float den = rho + rp;
            float delta = (den > 0.0f) ? (am * (rho + x1) + bm * bm) / den : 0.0f;
            float vr2 = vnx, vt2 = vny;
            if (rp > 0.0f) {
                float inv = one / rp;
                float ca = x1 * inv, sa = bm * inv;
                vr2 = ca * vnx + sa * vny;
                vt2 = ca * vny - sa * vnx;
            }
            float drn = dr + delta;
            float dzn = dz + cm;
            // carries beyond +-2^20 cells only occur for particles that leave the
            // domain; clamping keeps the integer conversion defined
            float kr = fminf(fmaxf(floorf(drn), -1048576.0f), 1048576.0f);
            drn = drn - kr;
            int ir2 = ir + (int)kr;
            if (drn >= one) {
                drn = drn - one;
                ir2 += 1;
            }
            float kz = fminf(fmaxf(floorf(dzn), -1048576.0f), 1048576.0f);
            dzn = dzn - kz;
            int iz2 = iz + (int)kz;
            if (dzn >= one) {
                dzn = dzn - one;
                iz2 += 1;
            }
            if (ir2 < 0) {
                ir2 = 0;
                drn = 0.0f;
            }
            // boundaries: electrode z < 0, wall r >= R, window z >= z_win
            bool he = iz2 < 0;
            bool hw = !he && ir2 >= nr;
            bool hd = !he && !hw && iz2 >= a.i_win;
            bool emit = false;
            if (sp == 1 && S.see_g > 0.0f && (he || hw || hd))
                emit = see_emit(cc, step, S, s_uid[p], he ? 0 : (hw ? 1 : 2), (uint32_t)(iz * nr + ir), dr, dz,
                                wrel);
            if (hd) {
                const float qd = emit ? wq * 2.0f : wq;
                float rpos = (float)ir2 + drn;
                int j0 = (int)floorf(rpos);
                float fr = rpos - (float)j0;
                atomicAdd(&a.win[a.i_win * NR + j0], (double)(qd * (one - fr)));
                atomicAdd(&a.win[a.i_win * NR + min(j0 + 1, nr)], (double)(qd * fr));
            }
            const bool alive = !(he || hw || hd);
            uint32_t ncell = kDead;
            if (alive) {
                ncell = (uint32_t)(iz2 * nr + ir2);
                float wa2 = one - drn, wb2 = one - dzn;
                dep_home(dq, dq2, tq, iz2, ir2, wq * (wa2 * wb2), wq * (drn * wb2), wq * (wa2 * dzn),
                         wq * (drn * dzn));
                // null-collision test; candidates are processed densely below
                if (u01(rnull) < S.pnull) {
                    int slot = atomicAdd(&s_ncand, 1);
                    s_cand[slot] = (uint16_t)p;
                }
            } else {
                ++cnt[1 + sp];
            }
            s_cell[p] = ncell;
            s_dr[p] = alive ? drn : 0.0f;
            s_dz[p] = alive ? dzn : 0.0f;
            s_vr[p] = vr2;
            s_vt[p] = vt2;
            s_vz[p] = vnz;
        }
        dep_flush_warp(dj, tj);
        if (dq2.iz >= 0) tile_add4(tq, dq2.iz, dq2.ir, dq2.v0, dq2.v1, dq2.v2, dq2.v3);
        dep_flush_warp(dq, tq);
        __syncthreads();
        // ---- phase B: collisions of the candidates
        const int nc = s_ncand;
        if (t < nc) {
            unsigned pc[6] = {0, 0, 0, 0, 0, 0};
            for (int c = t; c < nc; c += kPushThreads) {
                const int p = s_cand[c];
                float vx = s_vr[p], vy = s_vt[p], vzz = s_vz[p];
                if (sp == 0)
                    electron_collision(cc, step, S, s_uid[p], vx, vy, vzz, s_cell[p], s_dr[p], s_dz[p], pc,
                                       W ? __ldg(P.w + base + p) : 1.0f);
                else
                    ion_collision(cc, step, S, s_uid[p], vx, vy, vzz, pc);
                s_vr[p] = vx;
                s_vt[p] = vy;
                s_vz[p] = vzz;
            }
            for (int q = 0; q < 6; ++q)
                if (pc[q]) atomicAdd(&s_pc[q], pc[q]);
        }
        __syncthreads();
        // ---- write back (bulk) and flush the node tiles
        if (t == 0) {
            fence_async_smem();
            bulk_s2g(P.cell + base, s_cell, bytes);
            bulk_s2g(P.dr + base, s_dr, bytes);
            bulk_s2g(P.dz + base, s_dz, bytes);
            bulk_s2g(P.vr + base, s_vr, bytes);
            bulk_s2g(P.vt + base, s_vt, bytes);
            bulk_s2g(P.vz + base, s_vz, bytes);
            bulk_commit();
        }
        // warp w flushes and clears tile row w (trows <= kTileRows = warps per block)
        if (warp < trows)
            for (int cq = lane; cq < tcols; cq += 32) {
                const int q = warp * tcols + cq;
                const float vq = t_rho[q], vj = t_jm[q];
                t_rho[q] = 0.f;
                t_jm[q] = 0.f;
                const int gidx = (tlo + warp) * NR + tclo + cq;
                if (vq != 0.f) atomicAdd(&rho_sp[gidx], vq);
                if (vj != 0.f) atomicAdd(&a.jm[gidx], vj);
            }
        // every thread read this chunk's index before the barrier after the
        // tile bounds, so it can be replaced here
        if (t == 0) s_chunk = atomicAdd(&a.st->push_chunk, 1);
        __syncthreads();
    }
    if (t == 0) bulk_wait_all();
    // ---- block reduction of the tallies
    for (int o = 16; o > 0; o >>= 1) {
        acc_ind += __shfl_xor_sync(0xffffffffu, acc_ind, o);
        acc_es += __shfl_xor_sync(0xffffffffu, acc_es, o);
    }
    for (int q = 0; q < 3; ++q) cnt[q] = __reduce_add_sync(0xffffffffu, cnt[q]);
    if (lane == 0) {
        s_f[warp][0] = acc_ind;
        s_f[warp][1] = acc_es;
        for (int q = 0; q < 3; ++q) s_c[warp][q] = cnt[q];
    }
    __syncthreads();
    if (t == 0) {
        double si = 0, se = 0;
        // 0 el/cx, 1 ex/iso, 2 iz, 3 cx, 4 iso, 5 nu violations, 6 pushed, 7 absorbed e, 8 absorbed i
        unsigned long long tot[10] = {s_pc[0], s_pc[1], s_pc[2], s_pc[3], s_pc[4], s_pc[5], 0, 0, 0, 0};
        for (int w = 0; w < kPushThreads / 32; ++w) {
            si += s_f[w][0];
            se += s_f[w][1];
            for (int q = 0; q < 3; ++q) tot[6 + q] += s_c[w][q];
        }
        DevState* st = a.st;
        atomicAdd(&st->p_ind_step, si);
        atomicAdd(&st->p_es_step, se);
        // electron processes in 0..2, ion processes in 3..4
        const int map[7] = {C_E_EL, C_E_EX, C_E_IZ, C_I_CX, C_I_ISO, C_NUVIOL, C_PSTEPS};
        for (int q = 0; q < 7; ++q)
            if (tot[q]) {
                atomicAdd(&st->cnt[map[q]], tot[q]);
                atomicAdd(&st->per[map[q]], tot[q]);
            }
        unsigned long long ab = tot[7] + tot[8];
        if (ab) {
            atomicAdd(&st->cnt[C_ABSORBED], ab);
            atomicAdd(&st->per[C_ABSORBED], ab);
        }
        if (tot[7]) atomicAdd(&st->live[0], (unsigned long long)(-(long long)tot[7]));
        if (tot[8]) atomicAdd(&st->live[1], (unsigned long long)(-(long long)tot[8]));
    }
}

using PushFn = void (*)(PushArgs);

static int push_ppt(const Cell* c) { return c->push_ppt > 0 ? c->push_ppt : kPPT; }

template <bool W, bool IMPL>
static PushFn push_fn_w(int ppt) {
    switch (ppt) {
        case 4: return push_kernel<W, 4, IMPL>;
        case 16: return push_kernel<W, 16, IMPL>;
        default: return push_kernel<W, 8, IMPL>;
    }
}

static PushFn push_fn(const Cell* c) {
    const int ppt = push_ppt(c);
    if (c->implicit) return c->weighted ? push_fn_w<true, true>(ppt) : push_fn_w<false, true>(ppt);
    return c->weighted ? push_fn_w<true, false>(ppt) : push_fn_w<false, false>(ppt);
}

void push_prepare(Cell* c) {
    if (c->push_blocks) return;
    const size_t shm = PushSmem::bytes(c->NR, push_ppt(c));
    const PushFn fn = push_fn(c);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    int dev = 0, nsm = 148, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kPushThreads, shm);
    per = per < 1 ? 1 : per;
    c->push_per_sm_max = per;
    c->push_blocks = nsm * ((c->push_per_sm > 0 && c->push_per_sm < per) ? c->push_per_sm : per);
}

void launch_push(Cell* c, cudaStream_t st) {
    PushArgs a;
    for (int s = 0; s < 2; ++s) {
        a.p[s] = c->pb[s][c->cur[s]];
        a.sp[s] = c->sc[s];
    }
    a.nslot = c->d_nslot;
    a.F = c->d_F;
    a.rho[0] = c->d_rho;
    a.rho[1] = c->d_rho + c->nnodes;
    a.implicit = c->implicit ? 1 : 0;
    a.jm = c->d_jm;
    a.win = c->d_win;
    a.nr = c->nr;
    a.NR = c->NR;
    a.i_win = c->i_win;
    a.div_magic = c->div_magic;
    a.div_shift = c->div_shift;
    a.step = &c->d_st->step;
    a.key0 = (uint32_t)(c->cfg.seed & 0xffffffffu);
    a.key1 = (uint32_t)(c->cfg.seed >> 32);
    a.ev = c->d_events;
    a.ev_cap = c->event_cap;
    a.st = c->d_st;
    const size_t shm = PushSmem::bytes(c->NR, push_ppt(c));
    push_prepare(c);
    push_fn(c)<<<c->push_blocks, kPushThreads, shm, st>>>(a);
    count_launch();
}

// ---------------------------------------------------------------- bounded waits, self-test
// The two kinds of wait the library's kernels use, each on a condition that
// never comes true, so that their expiry path runs: an mbarrier phase that no
// copy completes (the particle kernel's staging wait) and a flag in global
// memory that no one sets, read with acquire loads (the shape of the cluster
// solve's barrier).  Each gives up after max_iters polls and records
// PP_ST_TIMEOUT in *status; nothing faults and the context stays usable.
__global__ void wait_selftest_kernel(long long max_iters, const unsigned* flag, unsigned* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const uint32_t addr = smem_u32(&bar);
    bool done = false;
    for (long long it = 0; it < max_iters && !done; ++it) {
        uint32_t d;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(d)
            : "r"(addr), "r"(0u)
            : "memory");
        done = d != 0;
    }
    if (!done) atomicOr(status, (unsigned)PP_ST_TIMEOUT);
    bool seen = false;
    for (long long it = 0; it < max_iters && !seen; ++it) {
        unsigned v;
        asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        seen = v != 0u;
    }
    if (!seen) atomicOr(status + 1, (unsigned)PP_ST_TIMEOUT);
}

int wait_selftest(long long max_iters, unsigned* status_out) {
    unsigned* d = nullptr;
    if (cudaMalloc(&d, 3 * sizeof(unsigned)) != cudaSuccess) return PP_E_CUDA;
    cudaMemset(d, 0, 3 * sizeof(unsigned));
    wait_selftest_kernel<<<1, 32>>>(max_iters, d + 2, d);
    count_launch();
    unsigned h[2] = {0u, 0u};
    cudaError_t e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return PP_E_CUDA;
    status_out[0] = h[0];
    status_out[1] = h[1];
    return PP_OK;
}

// ---------------------------------------------------------------- prime deposit
template <typename T>
__global__ void deposit_only(PBuf<T> P, const int* nslot, int sp, T qw, T* rho, int nr, int NR) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nslot[sp]) return;
    uint32_t cell = P.cell[idx];
    if (cell == kDead) return;
    int iz = (int)(cell / (uint32_t)nr), ir = (int)(cell - (uint32_t)iz * (uint32_t)nr);
    T dr = P.dr[idx], dz = P.dz[idx];
    T wa = T(1.0) - dr, wb = T(1.0) - dz;
    const T q = P.w ? qw * P.w[idx] : qw;
    T* p = rho + iz * NR + ir;
    atomicAdd(p, q * (wa * wb));
    atomicAdd(p + 1, q * (dr * wb));
    atomicAdd(p + NR, q * (wa * dz));
    atomicAdd(p + NR + 1, q * (dr * dz));
}

void launch_deposit_only(Cell* c, cudaStream_t st) {
    for (int s = 0; s < 2; ++s) {
        int64_t n = c->cap[s];
        unsigned nb = (unsigned)((n + 255) / 256);
        if (c->fp64)
            deposit_only<double><<<nb, 256, 0, st>>>(c->pd[s][c->cur[s]], c->d_nslot, s, c->scd[s].qw,
                                                     c->d_rho64 + (size_t)s * c->nnodes,
                                                     c->nr, c->NR);
        else
            deposit_only<float><<<nb, 256, 0, st>>>(c->pb[s][c->cur[s]], c->d_nslot, s, c->sc[s].qw,
                                                    c->d_rho + (size_t)s * c->nnodes,
                                                    c->nr, c->NR);
        count_launch();
    }
}

// ---------------------------------------------------------------- append events
// The step's creation events are appended in (kind, parent uid) order:
// ionisations (kind 0) as e- / Ar+ pairs, then secondary emissions (kind 1)
// as electrons.  A new particle's uid is next_uid + its rank among its
// species' new particles (a parent ionises at most once per step and an ion
// is absorbed once, so the keys are distinct and an event's rank is the
// number of events with a smaller key).  Block b ranks events
// [b*kAppendThreads, (b+1)*kAppendThreads) against all events, staged through
// shared memory in tiles, and scatters their indices into `perm`; the last
// block to finish (arrival counter, no waiting) writes the particles and
// updates the slot counts, uids and counters.  The grid covers the event
// capacity; blocks beyond the step's event count return at once.
template <typename T>
__global__ void __launch_bounds__(kAppendThreads) append_kernel(PBuf<T> pe, PBuf<T> pi, int* nslot,
                                                                uint32_t* next_uid, const EventT<T>* ev,
                                                                uint32_t* perm, int ev_cap, DevState* st,
                                                                int64_t cap_e, int64_t cap_i) {
    constexpr int kTile = 4096;
    __shared__ unsigned long long tile[kTile];
    __shared__ int s_last;
    const int n_ev = min(st->n_events, ev_cap);
    const int first = blockIdx.x * kAppendThreads;
    if (n_ev == 0 || first >= n_ev) return;
    const int nblk = (n_ev + kAppendThreads - 1) / kAppendThreads;
    const int q = first + (int)threadIdx.x;
    const unsigned long long kq =
        (q < n_ev) ? (((unsigned long long)ev[q].kind << 32) | (unsigned long long)ev[q].parent) : 0ull;
    int rank = 0;
    for (int base = 0; base < n_ev; base += kTile) {
        const int m = min(kTile, n_ev - base);
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += kAppendThreads)
            tile[j] = ((unsigned long long)ev[base + j].kind << 32) | (unsigned long long)ev[base + j].parent;
        __syncthreads();
        if (q < n_ev)
            for (int j = 0; j < m; ++j) rank += tile[j] < kq ? 1 : 0;
    }
    if (q < n_ev) perm[rank] = (uint32_t)q;
    // the last block to arrive sees every rank
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&st->append_done, 1) == nblk - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int ne = nslot[0], ni = nslot[1];
    const int n_see = min(((volatile int*)&st->n_see)[0], n_ev);
    const int n_pair = n_ev - n_see;
    int n_pair_add = n_pair;
    if ((int64_t)ne + n_pair_add > cap_e) n_pair_add = (int)(cap_e - ne);
    if ((int64_t)ni + n_pair_add > cap_i) n_pair_add = (int)(cap_i - ni);
    if (n_pair_add < 0) n_pair_add = 0;
    int n_see_add = 0;
    if (n_pair_add == n_pair) {
        n_see_add = n_see;
        if ((int64_t)ne + n_pair + n_see_add > cap_e) n_see_add = (int)(cap_e - ne - n_pair);
        if (n_see_add < 0) n_see_add = 0;
    }
    const int n_e_add = n_pair_add + n_see_add;
    const uint32_t ue = next_uid[0], ui = next_uid[1];
    for (int r = threadIdx.x; r < n_e_add; r += kAppendThreads) {
        const EventT<T> e = ev[((volatile uint32_t*)perm)[r]];
        pe.cell[ne + r] = e.cell;
        pe.dr[ne + r] = e.dr;
        pe.dz[ne + r] = e.dz;
        pe.vr[ne + r] = e.ve[0];
        pe.vt[ne + r] = e.ve[1];
        pe.vz[ne + r] = e.ve[2];
        pe.uid[ne + r] = ue + (uint32_t)r;
        if (pe.w) pe.w[ne + r] = e.w;
        if (r < n_pair_add) {
            pi.cell[ni + r] = e.cell;
            pi.dr[ni + r] = e.dr;
            pi.dz[ni + r] = e.dz;
            pi.vr[ni + r] = e.vi[0];
            pi.vt[ni + r] = e.vi[1];
            pi.vz[ni + r] = e.vi[2];
            pi.uid[ni + r] = ui + (uint32_t)r;
            if (pi.w) pi.w[ni + r] = e.w;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        nslot[0] = ne + n_e_add;
        nslot[1] = ni + n_pair_add;
        next_uid[0] = ue + (uint32_t)n_e_add;
        next_uid[1] = ui + (uint32_t)n_pair_add;
        st->cnt[C_CREATED] += (unsigned long long)n_pair_add;
        st->live[0] += (unsigned long long)n_e_add;
        st->live[1] += (unsigned long long)n_pair_add;
        st->per[C_CREATED] += (unsigned long long)n_pair_add;
        st->ctl[0] += (unsigned long long)n_see_add;
        if (n_e_add < n_ev) st->status |= PP_ST_CAPACITY;
        st->n_events = 0;
        st->n_see = 0;
        st->append_done = 0;
    }
}

void launch_append(Cell* c, cudaStream_t st) {
    const unsigned nb = (unsigned)((c->event_cap + kAppendThreads - 1) / kAppendThreads);
    if (c->fp64)
        append_kernel<double><<<nb, kAppendThreads, 0, st>>>(c->pd[0][c->cur[0]], c->pd[1][c->cur[1]], c->d_nslot,
                                                             c->d_next_uid, c->d_events64, c->d_ev_perm,
                                                             c->event_cap, c->d_st, c->cap[0], c->cap[1]);
    else
        append_kernel<float><<<nb, kAppendThreads, 0, st>>>(c->pb[0][c->cur[0]], c->pb[1][c->cur[1]], c->d_nslot,
                                                            c->d_next_uid, c->d_events, c->d_ev_perm, c->event_cap,
                                                            c->d_st, c->cap[0], c->cap[1]);
    count_launch();
}

// ---------------------------------------------------------------- counting sort
__global__ void sort_hist(const uint32_t* cell, const int* nslot, int sp, uint32_t* hist, int ncell) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = idx < nslot[sp];
    uint32_t c = act ? cell[idx] : kDead;
    int bin = (c == kDead) ? ncell : (int)c;
    unsigned peers = __match_any_sync(0xffffffffu, act ? bin : -1);
    int leader = __ffs(peers) - 1;
    if (act && (threadIdx.x & 31) == leader) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
}

// exclusive scan of n bins in one block; hist[n] receives the total
__global__ void sort_scan(uint32_t* hist, int n) {
    __shared__ uint32_t part[1024];
    int t = threadIdx.x;
    int per = (n + blockDim.x - 1) / blockDim.x;
    int lo = t * per, hi = min(lo + per, n);
    uint32_t s = 0;
    for (int q = lo; q < hi; ++q) s += hist[q];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        uint32_t v = (t >= o) ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = part[t] - s;
    for (int q = lo; q < hi; ++q) {
        uint32_t h = hist[q];
        hist[q] = run;
        run += h;
    }
    if (t == blockDim.x - 1) hist[n] = part[t];
}

template <typename T>
__global__ void sort_scatter(PBuf<T> src, PBuf<T> dst, const int* nslot, int sp, uint32_t* offs) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = idx < nslot[sp];
    uint32_t c = act ? src.cell[idx] : kDead;
    act = act && c != kDead;
    int key = act ? (int)c : -1;
    unsigned peers = __match_any_sync(0xffffffffu, key);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (act && lane == leader) base = atomicAdd(&offs[c], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!act) return;
    uint32_t pos = base + __popc(peers & ((1u << lane) - 1u));
    dst.cell[pos] = c;
    dst.dr[pos] = src.dr[idx];
    dst.dz[pos] = src.dz[idx];
    dst.vr[pos] = src.vr[idx];
    dst.vt[pos] = src.vt[idx];
    dst.vz[pos] = src.vz[idx];
    dst.uid[pos] = src.uid[idx];
    if (src.w) dst.w[pos] = src.w[idx];
}

// the new slot count, then the bins are cleared for the next sort
__global__ void sort_finish(int* nslot, int sp, uint32_t* hist, int ncell) {
    __shared__ uint32_t total;
    if (threadIdx.x == 0) total = hist[ncell];
    __syncthreads();
    if (threadIdx.x == 0) nslot[sp] = (int)total;
    for (int q = threadIdx.x; q < ncell + 2; q += blockDim.x) hist[q] = 0u;
}

void launch_sort(Cell* c, int sp, cudaStream_t st) {
    int ncell = c->i_win * c->nr;
    int64_t n = c->cap[sp];
    unsigned nb = (unsigned)((n + 255) / 256);
    const uint32_t* src_cell = c->fp64 ? c->pd[sp][c->cur[sp]].cell : c->pb[sp][c->cur[sp]].cell;
    sort_hist<<<nb, 256, 0, st>>>(src_cell, c->d_nslot, sp, c->d_hist, ncell);
    // live bins only: the dead bin (index ncell) is left out of the scan
    sort_scan<<<1, 1024, 0, st>>>(c->d_hist, ncell);
    if (c->fp64)
        sort_scatter<double><<<nb, 256, 0, st>>>(c->pd[sp][c->cur[sp]], c->pd[sp][1 - c->cur[sp]], c->d_nslot, sp,
                                                 c->d_hist);
    else
        sort_scatter<float><<<nb, 256, 0, st>>>(c->pb[sp][c->cur[sp]], c->pb[sp][1 - c->cur[sp]], c->d_nslot, sp,
                                                c->d_hist);
    sort_finish<<<1, 1024, 0, st>>>(c->d_nslot, sp, c->d_hist, ncell);
    count_launch(4);
    c->cur[sp] = 1 - c->cur[sp];
}

}  // namespace pp
