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

#include <climits>

namespace pp {

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: round (c0..c3; k0,k1) -> (hi(M1 c2)^c1^k0, lo(M1 c2),
// hi(M0 c0)^c3^k1, lo(M0 c0)), key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// ((x >> 9) + 0.5) * 2^-23, exact in float32, in (0, 1)
__device__ __forceinline__ float u01(uint32_t x) {
    return (float)(int)(((x >> 9) << 1) | 1u) * 5.9604644775390625e-8f;
}

struct U4 {
    float a, b, c, d;
};

__device__ __forceinline__ U4 draw4(uint32_t uid, uint32_t step, uint32_t call, uint32_t sp, uint32_t k0,
                                    uint32_t k1) {
    uint4 r = philox4x32_10(make_uint4(uid, step, call, sp), k0, k1);
    return U4{u01(r.x), u01(r.y), u01(r.z), u01(r.w)};
}

// ---------------------------------------------------------------- cross sections
// electron-Ar (units 1e-20 m^2) at energy x (eV); project-defined rational fits
__device__ __forceinline__ void sigma_e(float x, float& el, float& ex, float& iz) {
    float y = x - 0.23f;
    float y2 = y * y;
    el = (0.1f + 14.0f * y2 / (y2 + 4.0f)) / (1.0f + x / 50.0f);
    float ye = x - kEExc;
    ex = (x > kEExc) ? 1.2f * ye / (ye * ye / 30.0f + ye + 8.0f) : 0.0f;
    float yi = x - kEIon;
    iz = (x > kEIon) ? 3.0f * yi / (yi * yi / 60.0f + yi + 30.0f) : 0.0f;
}

// Ar+-Ar charge exchange and isotropic elastic (units 1e-19 m^2) at lab energy x
__device__ __forceinline__ void sigma_i(float x, float& cx, float& iso) {
    float sq = sqrtf(x);
    cx = 2.0f + 3.0f / (1.0f + sq);
    iso = 1.0f + 2.0f / (1.0f + sq);
}

__device__ __forceinline__ void iso_dir(float u2, float u3, float& dx, float& dy, float& dz) {
    float c = 1.0f - 2.0f * u2;
    float s = sqrtf(fmaxf(1.0f - c * c, 0.0f));
    float sp, cp;
    sincospif(2.0f * u3, &sp, &cp);
    dx = s * cp;
    dy = s * sp;
    dz = c;
}

__device__ __forceinline__ void gauss3(float a, float b, float c, float d, float& n0, float& n1, float& n2) {
    float ra = sqrtf(-2.0f * logf(a));
    float rc = sqrtf(-2.0f * logf(c));
    float sb, cb, sd, cd;
    sincospif(2.0f * b, &sb, &cb);
    sincospif(2.0f * d, &sd, &cd);
    n0 = ra * cb;
    n1 = ra * sb;
    n2 = rc * cd;
}

// ---------------------------------------------------------------- deposition
struct Tile {
    float* s;      // shared rows [lo, lo + rows)
    int lo, rows;
    float* g;      // global node grid
    int NR;
};

__device__ __forceinline__ void add4(const Tile& t, int iz, int ir, float v0, float v1, float v2, float v3) {
    int r0 = iz - t.lo;
    if (r0 >= 0 && r0 + 1 < t.rows) {
        float* p = t.s + r0 * t.NR + ir;
        atomicAdd(p, v0);
        atomicAdd(p + 1, v1);
        atomicAdd(p + t.NR, v2);
        atomicAdd(p + t.NR + 1, v3);
    } else {
        float* p = t.g + iz * t.NR + ir;
        atomicAdd(p, v0);
        atomicAdd(p + 1, v1);
        atomicAdd(p + t.NR, v2);
        atomicAdd(p + t.NR + 1, v3);
    }
}

// Warp-aggregated bilinear deposit: the largest group of lanes that share a
// cell is summed by a butterfly and written once; the other lanes add their
// own four values.  All 32 lanes must call it.
__device__ __forceinline__ void deposit4(bool act, int iz, int ir, float v0, float v1, float v2, float v3,
                                         const Tile& t) {
    const unsigned full = 0xffffffffu;
    int lane = threadIdx.x & 31;
    int key = act ? iz * t.NR + ir : -1;
    unsigned peers = __match_any_sync(full, key);
    int leader = __ffs(peers) - 1;
    unsigned gsize = __popc(peers);
    unsigned code = act ? ((gsize << 5) | (unsigned)(31 - leader)) : 0u;
    unsigned best = __reduce_max_sync(full, code);
    bool agg = false;
    if ((best >> 5) >= 2u) {
        int bl = 31 - (int)(best & 31u);
        agg = act && (leader == bl);
        float s0 = agg ? v0 : 0.f, s1 = agg ? v1 : 0.f, s2 = agg ? v2 : 0.f, s3 = agg ? v3 : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(full, s0, o);
            s1 += __shfl_xor_sync(full, s1, o);
            s2 += __shfl_xor_sync(full, s2, o);
            s3 += __shfl_xor_sync(full, s3, o);
        }
        if (lane == bl) add4(t, iz, ir, s0, s1, s2, s3);
    }
    if (act && !agg) add4(t, iz, ir, v0, v1, v2, v3);
}

// ---------------------------------------------------------------- push kernel
struct PushArgs {
    ParticleBuf p[2];
    const int* nslot;
    SpeciesConst sp[2];
    const float* F;
    float* rho;
    float* jm;
    double* win;
    int nr, NR, i_win;
    uint32_t step, key0, key1;
    Event* ev;
    DevState* st;
};

__global__ void __launch_bounds__(kPushThreads) push_kernel(PushArgs a) {
    __shared__ float t_rho[kTileRows * kMaxNR];
    __shared__ float t_jm[kTileRows * kMaxNR];
    __shared__ int s_min[kPushThreads / 32], s_max[kPushThreads / 32];
    __shared__ float s_f[kPushThreads / 32][2];
    __shared__ unsigned s_c[kPushThreads / 32][9];

    const int n0 = a.nslot[0], n1 = a.nslot[1];
    const int ce = (n0 + kChunk - 1) / kChunk, ci = (n1 + kChunk - 1) / kChunk;
    const int nr = a.nr, NR = a.NR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float acc_ind = 0.f, acc_es = 0.f;
    unsigned c_push = 0, c_abs = 0, c_abs1 = 0, c_el = 0, c_ex = 0, c_iz = 0, c_cx = 0, c_iso = 0, c_viol = 0;

    for (int chunk = blockIdx.x; chunk < ce + ci; chunk += gridDim.x) {
        const int sp = chunk < ce ? 0 : 1;
        const int base = (chunk - (sp ? ce : 0)) * kChunk;
        const int n = sp ? n1 : n0;
        const ParticleBuf P = a.p[sp];
        const SpeciesConst S = a.sp[sp];

        uint32_t cells[kPPT];
        int lmin = INT_MAX, lmax = -1;
#pragma unroll
        for (int k = 0; k < kPPT; ++k) {
            int idx = base + k * kPushThreads + threadIdx.x;
            cells[k] = (idx < n) ? P.cell[idx] : kDead;
            if (cells[k] != kDead) {
                int iz = (int)(cells[k] / (uint32_t)nr);
                lmin = min(lmin, iz);
                lmax = max(lmax, iz);
            }
        }
        lmin = __reduce_min_sync(0xffffffffu, lmin);
        lmax = __reduce_max_sync(0xffffffffu, lmax);
        if (lane == 0) {
            s_min[warp] = lmin;
            s_max[warp] = lmax;
        }
        __syncthreads();
        int bmin = INT_MAX, bmax = -1;
        for (int w = 0; w < kPushThreads / 32; ++w) {
            bmin = min(bmin, s_min[w]);
            bmax = max(bmax, s_max[w]);
        }
        int tlo = max(bmin - 1, 0);
        int thi = min(bmax + 2, a.i_win);
        int trows = (bmax < 0) ? 0 : min(thi - tlo + 1, kTileRows);
        for (int q = threadIdx.x; q < trows * NR; q += kPushThreads) {
            t_rho[q] = 0.f;
            t_jm[q] = 0.f;
        }
        __syncthreads();
        Tile tj{t_jm, tlo, trows, a.jm, NR};
        Tile tq{t_rho, tlo, trows, a.rho, NR};

#pragma unroll 1
        for (int k = 0; k < kPPT; ++k) {
            const int idx = base + k * kPushThreads + threadIdx.x;
            const bool live = cells[k] != kDead;
            int iz = 0, ir = 0;
            float dr = 0.f, dz = 0.f, vr = 0.f, vt = 0.f, vz = 0.f;
            uint32_t uid = 0;
            if (live) {
                iz = (int)(cells[k] / (uint32_t)nr);
                ir = (int)(cells[k] - (uint32_t)iz * (uint32_t)nr);
                dr = P.dr[idx];
                dz = P.dz[idx];
                vr = P.vr[idx];
                vt = P.vt[idx];
                vz = P.vz[idx];
                uid = P.uid[idx];
            }
            // ---- gather (bilinear weights at the old position)
            const float one = 1.0f;
            float wa = one - dr, wb = one - dz;
            float w00 = wa * wb, w01 = dr * wb, w10 = wa * dz, w11 = dr * dz;
            float Er = 0.f, Ez = 0.f, Et = 0.f, Br = 0.f, Bz = 0.f;
            if (live) {
                const float4* f = reinterpret_cast<const float4*>(a.F) + (size_t)cells[k] * 5;
                float4 q0 = __ldg(f), q1 = __ldg(f + 1), q2 = __ldg(f + 2), q3 = __ldg(f + 3), q4 = __ldg(f + 4);
                Er = w00 * q0.x + w01 * q0.y + w10 * q0.z + w11 * q0.w;
                Ez = w00 * q1.x + w01 * q1.y + w10 * q1.z + w11 * q1.w;
                Et = w00 * q2.x + w01 * q2.y + w10 * q2.z + w11 * q2.w;
                Br = w00 * q3.x + w01 * q3.y + w10 * q3.z + w11 * q3.w;
                Bz = w00 * q4.x + w01 * q4.y + w10 * q4.z + w11 * q4.w;
            }
            // ---- Boris in the local frame (x = r, y = theta, z); B_theta = 0
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
            // ---- current moment at the old position, time-centred velocity
            float vbt = (vt + vny) * 0.5f;
            float vbr = (vr + vnx) * 0.5f;
            float vbz = (vz + vnz) * 0.5f;
            float jmv = S.qw * vbt;
            if (live) {
                acc_ind += jmv * Et;
                acc_es += S.qw * (vbr * Er + vbz * Ez);
                ++c_push;
            }
            deposit4(live, iz, ir, jmv * w00, jmv * w01, jmv * w10, jmv * w11, tj);
            // ---- move (cell units); r' = |(r + a, b)| written as r + delta
            float am = vnx * S.dtr, bm = vny * S.dtr, cm = vnz * S.dtz;
            float rho = (float)ir + dr;
            float x1 = rho + am;
            float rp = sqrtf(x1 * x1 + bm * bm);
            float den = rho + rp;
            float delta = (den > 0.0f) ? (am * (rho + x1) + bm * bm) / den : 0.0f;
            float vr2 = vnx, vt2 = vny;
            if (rp > 0.0f) {
                float ca = x1 / rp, sa = bm / rp;
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
            // ---- boundaries: electrode z < 0, wall r >= R, window z >= z_win
            bool alive = live;
            if (live) {
                bool he = iz2 < 0;
                bool hw = !he && ir2 >= nr;
                bool hd = !he && !hw && iz2 >= a.i_win;
                if (hd) {
                    float rpos = (float)ir2 + drn;
                    int j0 = (int)floorf(rpos);
                    float fr = rpos - (float)j0;
                    atomicAdd(&a.win[a.i_win * NR + j0], (double)(S.qw * (one - fr)));
                    atomicAdd(&a.win[a.i_win * NR + min(j0 + 1, nr)], (double)(S.qw * fr));
                }
                if (he || hw || hd) {
                    alive = false;
                    ++c_abs;
                    if (sp) ++c_abs1;
                }
            }
            // ---- null-collision MCC at the new position
            float ovr = vr2, ovt = vt2, ovz = vnz;
            if (alive) {
                U4 u = draw4(uid, a.step, 0u, (uint32_t)sp, a.key0, a.key1);
                if (u.a < S.pnull) {
                    float x = vr2, y = vt2, z = vnz;
                    if (sp == 0) {
                        float v2 = x * x + y * y + z * z;
                        float g = sqrtf(v2);
                        float en = v2 * S.ce;
                        float s_el, s_ex, s_iz;
                        sigma_e(en, s_el, s_ex, s_iz);
                        float nu_el = S.ng * s_el * g;
                        float nu_ex = S.ng * s_ex * g;
                        float nu_iz = S.ng * s_iz * g;
                        float r = u.b * S.numax;
                        float c1 = nu_el, c2 = c1 + nu_ex, c3 = c2 + nu_iz;
                        if (c3 > S.numax) ++c_viol;
                        int proc = (r < c1) ? 0 : (r < c2) ? 1 : (r < c3) ? 2 : 3;
                        if (proc < 3) {
                            float dx, dy, dzz;
                            iso_dir(u.c, u.d, dx, dy, dzz);
                            float gn;
                            if (proc == 0) {
                                float cosx = (g > 0.0f) ? (x * dx + y * dy + z * dzz) / g : 0.0f;
                                gn = g * sqrtf(one - S.loss * (one - cosx));
                                ++c_el;
                            } else if (proc == 1) {
                                gn = sqrtf(fmaxf(en - kEExc, 0.0f) * S.inv_ce);
                                ++c_ex;
                            } else {
                                float eh = fmaxf(en - kEIon, 0.0f) * 0.5f;
                                gn = sqrtf(eh * S.inv_ce);
                                ++c_iz;
                                U4 a1 = draw4(uid, a.step, 1u, 0u, a.key0, a.key1);
                                U4 b1 = draw4(uid, a.step, 2u, 0u, a.key0, a.key1);
                                float ex_, ey_, ez_, g0, g1, g2;
                                iso_dir(a1.a, a1.b, ex_, ey_, ez_);
                                gauss3(a1.c, a1.d, b1.a, b1.b, g0, g1, g2);
                                int slot = atomicAdd(&a.st->n_events, 1);
                                if (slot < kEventCap) {
                                    Event e;
                                    e.parent = uid;
                                    e.cell = (uint32_t)(iz2 * nr + ir2);
                                    e.dr = drn;
                                    e.dz = dzn;
                                    e.ve[0] = gn * ex_;
                                    e.ve[1] = gn * ey_;
                                    e.ve[2] = gn * ez_;
                                    e.vi[0] = a.sp[1].vth_gas * g0;
                                    e.vi[1] = a.sp[1].vth_gas * g1;
                                    e.vi[2] = a.sp[1].vth_gas * g2;
                                    a.ev[slot] = e;
                                } else {
                                    atomicOr(&a.st->status, (unsigned)PP_ST_EVENTS);
                                }
                            }
                            ovr = gn * dx;
                            ovt = gn * dy;
                            ovz = gn * dzz;
                        }
                    } else {
                        U4 a1 = draw4(uid, a.step, 1u, 1u, a.key0, a.key1);
                        float g0, g1, g2;
                        gauss3(a1.a, a1.b, a1.c, a1.d, g0, g1, g2);
                        float vnxn = S.vth_gas * g0, vnyn = S.vth_gas * g1, vnzn = S.vth_gas * g2;
                        float gx = x - vnxn, gy = y - vnyn, gz = z - vnzn;
                        float g2s = gx * gx + gy * gy + gz * gz;
                        float g = sqrtf(g2s);
                        float en = g2s * S.ce;
                        float s_cx, s_iso;
                        sigma_i(en, s_cx, s_iso);
                        float nu_cx = S.ng * s_cx * g;
                        float nu_iso = S.ng * s_iso * g;
                        float r = u.b * S.numax;
                        float c1 = nu_cx, c2 = c1 + nu_iso;
                        if (c2 > S.numax) ++c_viol;
                        if (r < c1) {
                            ovr = vnxn;
                            ovt = vnyn;
                            ovz = vnzn;
                            ++c_cx;
                        } else if (r < c2) {
                            float dx, dy, dzz;
                            iso_dir(u.c, u.d, dx, dy, dzz);
                            float hg = g * 0.5f;
                            ovr = (x + vnxn) * 0.5f + hg * dx;
                            ovt = (y + vnyn) * 0.5f + hg * dy;
                            ovz = (z + vnzn) * 0.5f + hg * dzz;
                            ++c_iso;
                        }
                    }
                }
            }
            // ---- charge at the new position
            float wa2 = one - drn, wb2 = one - dzn;
            float q00 = S.qw * (wa2 * wb2), q01 = S.qw * (drn * wb2), q10 = S.qw * (wa2 * dzn),
                  q11 = S.qw * (drn * dzn);
            deposit4(alive, iz2, ir2, q00, q01, q10, q11, tq);
            // ---- store
            if (live) {
                P.cell[idx] = alive ? (uint32_t)(iz2 * nr + ir2) : kDead;
                P.dr[idx] = alive ? drn : 0.0f;
                P.dz[idx] = alive ? dzn : 0.0f;
                P.vr[idx] = ovr;
                P.vt[idx] = ovt;
                P.vz[idx] = ovz;
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < trows * NR; q += kPushThreads) {
            float vq = t_rho[q], vj = t_jm[q];
            int gidx = (tlo + q / NR) * NR + (q % NR);
            if (vq != 0.f) atomicAdd(&a.rho[gidx], vq);
            if (vj != 0.f) atomicAdd(&a.jm[gidx], vj);
        }
        __syncthreads();
    }
    // ---- block reduction of the tallies
    for (int o = 16; o > 0; o >>= 1) {
        acc_ind += __shfl_xor_sync(0xffffffffu, acc_ind, o);
        acc_es += __shfl_xor_sync(0xffffffffu, acc_es, o);
    }
    unsigned cs[9] = {c_push, c_abs, c_el, c_ex, c_iz, c_cx, c_iso, c_viol, c_abs1};
    for (int q = 0; q < 9; ++q) cs[q] = __reduce_add_sync(0xffffffffu, cs[q]);
    if (lane == 0) {
        s_f[warp][0] = acc_ind;
        s_f[warp][1] = acc_es;
        for (int q = 0; q < 9; ++q) s_c[warp][q] = cs[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double si = 0, se = 0;
        unsigned long long tot[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < kPushThreads / 32; ++w) {
            si += s_f[w][0];
            se += s_f[w][1];
            for (int q = 0; q < 9; ++q) tot[q] += s_c[w][q];
        }
        DevState* st = a.st;
        atomicAdd(&st->p_ind_step, si);
        atomicAdd(&st->p_es_step, se);
        const int map[8] = {C_PSTEPS, C_ABSORBED, C_E_EL, C_E_EX, C_E_IZ, C_I_CX, C_I_ISO, C_NUVIOL};
        for (int q = 0; q < 8; ++q)
            if (tot[q]) {
                atomicAdd(&st->cnt[map[q]], tot[q]);
                atomicAdd(&st->per[map[q]], tot[q]);
            }
        unsigned long long a1 = tot[8], a0 = tot[1] - tot[8];
        if (a0) atomicAdd(&st->live[0], (unsigned long long)(-(long long)a0));
        if (a1) atomicAdd(&st->live[1], (unsigned long long)(-(long long)a1));
    }
}

void launch_push(Cell* c, uint32_t step, cudaStream_t st) {
    PushArgs a;
    for (int s = 0; s < 2; ++s) {
        a.p[s] = c->pb[s][c->cur[s]];
        a.sp[s] = c->sc[s];
    }
    a.nslot = c->d_nslot;
    a.F = c->d_F;
    a.rho = c->d_rho;
    a.jm = c->d_jm;
    a.win = c->d_win;
    a.nr = c->nr;
    a.NR = c->NR;
    a.i_win = c->i_win;
    a.step = step;
    a.key0 = (uint32_t)(c->cfg.seed & 0xffffffffu);
    a.key1 = (uint32_t)(c->cfg.seed >> 32);
    a.ev = c->d_events;
    a.st = c->d_st;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    push_kernel<<<nsm * 4, kPushThreads, 0, st>>>(a);
    count_launch();
}

// ---------------------------------------------------------------- prime deposit
__global__ void deposit_only(ParticleBuf P, const int* nslot, int sp, float qw, float* rho, int nr, int NR) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nslot[sp]) return;
    uint32_t cell = P.cell[idx];
    if (cell == kDead) return;
    int iz = (int)(cell / (uint32_t)nr), ir = (int)(cell - (uint32_t)iz * (uint32_t)nr);
    float dr = P.dr[idx], dz = P.dz[idx];
    float wa = 1.0f - dr, wb = 1.0f - dz;
    float* p = rho + iz * NR + ir;
    atomicAdd(p, qw * (wa * wb));
    atomicAdd(p + 1, qw * (dr * wb));
    atomicAdd(p + NR, qw * (wa * dz));
    atomicAdd(p + NR + 1, qw * (dr * dz));
}

void launch_deposit_only(Cell* c, cudaStream_t st) {
    for (int s = 0; s < 2; ++s) {
        int64_t n = c->cap[s];
        deposit_only<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c->pb[s][c->cur[s]], c->d_nslot, s,
                                                                 c->sc[s].qw, c->d_rho, c->nr, c->NR);
        count_launch();
    }
}

// ---------------------------------------------------------------- append events
// One block: sort this step's events by parent uid (bitonic, in shared
// memory) and append the e- / Ar+ pairs with uid = next_uid + rank.
__global__ void append_kernel(ParticleBuf pe, ParticleBuf pi, int* nslot, uint32_t* next_uid, const Event* ev,
                              DevState* st, int64_t cap_e, int64_t cap_i) {
    __shared__ uint32_t key[kEventCap];
    __shared__ uint16_t val[kEventCap];
    int n_ev = min(st->n_events, kEventCap);
    if (n_ev == 0) return;
    int P2 = 1;
    while (P2 < n_ev) P2 <<= 1;
    for (int q = threadIdx.x; q < P2; q += blockDim.x) {
        key[q] = (q < n_ev) ? ev[q].parent : 0xFFFFFFFFu;
        val[q] = (uint16_t)q;
    }
    __syncthreads();
    for (int k = 2; k <= P2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int q = threadIdx.x; q < P2; q += blockDim.x) {
                int l = q ^ j;
                if (l > q) {
                    bool up = (q & k) == 0;
                    uint32_t kq = key[q], kl = key[l];
                    if ((kq > kl) == up) {
                        key[q] = kl;
                        key[l] = kq;
                        uint16_t t = val[q];
                        val[q] = val[l];
                        val[l] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
    int ne = nslot[0], ni = nslot[1];
    int n_add = n_ev;
    if ((int64_t)ne + n_add > cap_e) n_add = (int)(cap_e - ne);
    if ((int64_t)ni + n_add > cap_i) n_add = (int)(cap_i - ni);
    if (n_add < 0) n_add = 0;
    uint32_t ue = next_uid[0], ui = next_uid[1];
    for (int r = threadIdx.x; r < n_add; r += blockDim.x) {
        const Event e = ev[val[r]];
        pe.cell[ne + r] = e.cell;
        pe.dr[ne + r] = e.dr;
        pe.dz[ne + r] = e.dz;
        pe.vr[ne + r] = e.ve[0];
        pe.vt[ne + r] = e.ve[1];
        pe.vz[ne + r] = e.ve[2];
        pe.uid[ne + r] = ue + (uint32_t)r;
        pi.cell[ni + r] = e.cell;
        pi.dr[ni + r] = e.dr;
        pi.dz[ni + r] = e.dz;
        pi.vr[ni + r] = e.vi[0];
        pi.vt[ni + r] = e.vi[1];
        pi.vz[ni + r] = e.vi[2];
        pi.uid[ni + r] = ui + (uint32_t)r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        nslot[0] = ne + n_add;
        nslot[1] = ni + n_add;
        next_uid[0] = ue + (uint32_t)n_add;
        next_uid[1] = ui + (uint32_t)n_add;
        st->cnt[C_CREATED] += (unsigned long long)n_add;
        st->live[0] += (unsigned long long)n_add;
        st->live[1] += (unsigned long long)n_add;
        st->per[C_CREATED] += (unsigned long long)n_add;
        if (n_add < n_ev) st->status |= PP_ST_CAPACITY;
        st->n_events = 0;
    }
}

void launch_append(Cell* c, cudaStream_t st) {
    append_kernel<<<1, 1024, 0, st>>>(c->pb[0][c->cur[0]], c->pb[1][c->cur[1]], c->d_nslot, c->d_next_uid,
                                      c->d_events, c->d_st, c->cap[0], c->cap[1]);
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

__global__ void sort_scatter(ParticleBuf src, ParticleBuf dst, const int* nslot, int sp, uint32_t* offs) {
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
}

__global__ void sort_finish(int* nslot, int sp, const uint32_t* hist, int ncell) {
    nslot[sp] = (int)hist[ncell];
}

void launch_sort(Cell* c, int sp, cudaStream_t st) {
    int ncell = c->i_win * c->nr;
    cudaMemsetAsync(c->d_hist, 0, sizeof(uint32_t) * (ncell + 2), st);
    int64_t n = c->cap[sp];
    unsigned nb = (unsigned)((n + 255) / 256);
    ParticleBuf src = c->pb[sp][c->cur[sp]], dst = c->pb[sp][1 - c->cur[sp]];
    sort_hist<<<nb, 256, 0, st>>>(src.cell, c->d_nslot, sp, c->d_hist, ncell);
    // live bins only: the dead bin (index ncell) is left out of the scan
    sort_scan<<<1, 1024, 0, st>>>(c->d_hist, ncell);
    sort_scatter<<<nb, 256, 0, st>>>(src, dst, c->d_nslot, sp, c->d_hist);
    sort_finish<<<1, 1, 0, st>>>(c->d_nslot, sp, c->d_hist, ncell);
    count_launch(4);
    c->cur[sp] = 1 - c->cur[sp];
}

}  // namespace pp
