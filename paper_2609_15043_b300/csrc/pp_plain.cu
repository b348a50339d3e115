// Plain form of the particle step (the comparison baseline of the fused FP32
// kernel): one thread per particle slot, state of type T loaded and stored
// straight from global memory, the five fields gathered from the per-cell
// corner table, current and charge deposited with global atomics, collisions
// handled inline by the thread that found them.  Instantiated with double it
// is the plain FP64 PIC step; every arithmetic expression is the fused
// kernel's (and the oracle's) in the same order, evaluated in T, including the
// per-particle weights and the secondary emission of absorbed ions.
#include "pp_internal.h"
#include "pp_mcc.cuh"

namespace pp {

template <typename T>
struct PlainArgs {
    PBuf<T> p[2];
    const int* nslot;
    SpecT<T> sp[2];
    const T* F;            // per plasma cell: (Er, Ez, Etheta, Br, Bz) x corners 00, 01, 10, 11
    T* rho[2];             // node charge of the step per species (C)
    T* jm;                 // node current moment (A m)
    double* win;           // window surface charge (C)
    int nr, NR, i_win;
    int implicit;          // direct-implicit electrostatics
    const unsigned long long* step;
    uint32_t key0, key1;
    EventT<T>* ev;
    int ev_cap;
    DevState* st;
};

template <typename T>
__device__ __forceinline__ void add4(T* g, int NR, int iz, int ir, T v0, T v1, T v2, T v3) {
    T* p = g + iz * NR + ir;
    atomicAdd(p, v0);
    atomicAdd(p + 1, v1);
    atomicAdd(p + NR, v2);
    atomicAdd(p + NR + 1, v3);
}

template <typename T>
__global__ void __launch_bounds__(256, 2) push_plain(PlainArgs<T> a) {
    __shared__ double s_f[8][2];
    __shared__ unsigned s_c[8][10];
    const int n0 = a.nslot[0], n1 = a.nslot[1];
    const int nr = a.nr, NR = a.NR;
    const uint32_t step = (uint32_t)(*a.step);
    const CollCtx<T> cc{a.key0, a.key1, a.ev, a.ev_cap, a.st, a.sp[1].vth_gas};
    const T one = T(1.0);
    double acc_ind = 0.0, acc_es = 0.0;
    // 0..4 processes, 5 nu violations, 6 pushed, 7 absorbed e, 8 absorbed i
    unsigned cnt[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n0 + n1; g += gridDim.x * blockDim.x) {
        const int sp = g < n0 ? 0 : 1;
        const int q = sp ? g - n0 : g;
        const PBuf<T> P = sp ? a.p[1] : a.p[0];
        const SpecT<T> S = sp ? a.sp[1] : a.sp[0];
        const uint32_t cell = P.cell[q];
        if (cell == kDead) continue;
        int iz = (int)(cell / (uint32_t)nr);
        int ir = (int)cell - iz * nr;
        T dr = P.dr[q], dz = P.dz[q];
        T vr = P.vr[q], vz = P.vz[q];
        const T vt = P.vt[q];
        const T wrel = P.w ? P.w[q] : one;
        const T wq = P.w ? S.qw * wrel : S.qw;               // the particle's charge
        const T* f = a.F + (size_t)cell * 20;
        // gather (bilinear weights at the old position)
        T wa = one - dr, wb = one - dz;
        T w00 = wa * wb, w01 = dr * wb, w10 = wa * dz, w11 = dr * dz;
        T Er = w00 * f[0] + w01 * f[1] + w10 * f[2] + w11 * f[3];
        T Ez = w00 * f[4] + w01 * f[5] + w10 * f[6] + w11 * f[7];
        T Et = w00 * f[8] + w01 * f[9] + w10 * f[10] + w11 * f[11];
        T Br = w00 * f[12] + w01 * f[13] + w10 * f[14] + w11 * f[15];
        T Bz = w00 * f[16] + w01 * f[17] + w10 * f[18] + w11 * f[19];
        ++cnt[6];
        if (a.implicit) {
            // the previous step's implicit kick at the predicted position
            // (the fused kernel's arithmetic in T)
            const T vrc = vr + S.qmd * Er, vzc = vz + S.qmd * Ez;
            T tr = dr + S.kres * Er, tz = dz + S.kzes * Ez;
            T kr = fmin_t(fmax_t(floor_t(tr), T(-1048576.0)), T(1048576.0));
            tr = tr - kr;
            int irc = ir + (int)kr;
            if (tr >= one) {
                tr = tr - one;
                irc += 1;
            }
            T kz = fmin_t(fmax_t(floor_t(tz), T(-1048576.0)), T(1048576.0));
            tz = tz - kz;
            int izc = iz + (int)kz;
            if (tz >= one) {
                tz = tz - one;
                izc += 1;
            }
            T vr_k = vrc;
            if (irc < 0) {
                const T rpos = -((T)irc + tr);
                const T jf = floor_t(rpos);
                irc = (int)jf;
                tr = rpos - jf;
                vr_k = -vrc;
            }
            const bool ce = izc < 0;
            const bool cw = !ce && irc >= nr;
            const bool cd = !ce && !cw && izc >= a.i_win;
            if (ce || cw || cd) {
                bool emit = false;
                if (sp == 1 && S.see_g > T(0.0))
                    emit = see_emit(cc, step, S, P.uid[q], ce ? 0 : (cw ? 1 : 2), cell, dr, dz, wrel);
                if (cd) {
                    const T qd = emit ? wq * T(2.0) : wq;
                    T rpos = (T)irc + tr;
                    int j0 = (int)floor_t(rpos);
                    T fr = rpos - (T)j0;
                    atomicAdd(&a.win[a.i_win * NR + j0], (double)(qd * (one - fr)));
                    atomicAdd(&a.win[a.i_win * NR + min(j0 + 1, nr)], (double)(qd * fr));
                }
                ++cnt[7 + sp];
                P.cell[q] = kDead;
                P.dr[q] = T(0.0);
                P.dz[q] = T(0.0);
                continue;
            }
            acc_es += (double)(wq * (((vr + vrc) * T(0.5)) * Er + ((vz + vzc) * T(0.5)) * Ez));
            ir = irc;
            iz = izc;
            dr = tr;
            dz = tz;
            vr = vr_k;
            vz = vzc;
            wa = one - dr;
            wb = one - dz;
            w00 = wa * wb;
            w01 = dr * wb;
            w10 = wa * dz;
            w11 = dr * dz;
            Er = T(0.0);
            Ez = T(0.0);
        }
        // Boris in the local frame (x = r, y = theta, z); B_theta = 0
        T hx = S.qmh * Er, hy = S.qmh * Et, hz = S.qmh * Ez;
        T vmx = vr + hx, vmy = vt + hy, vmz = vz + hz;
        T tx = S.qmh * Br, tz = S.qmh * Bz;
        T t2 = tx * tx + tz * tz;
        T sf = T(2.0) / (one + t2);
        T sx = tx * sf, sz = tz * sf;
        T v1x = vmx + vmy * tz;
        T v1y = vmy + (vmz * tx - vmx * tz);
        T v1z = vmz - vmy * tx;
        T vpx = vmx + v1y * sz;
        T vpy = vmy + (v1z * sx - v1x * sz);
        T vpz = vmz - v1y * sx;
        T vnx = vpx + hx, vny = vpy + hy, vnz = vpz + hz;
        // current moment at the old position, time-centred velocity
        T vbt = (vt + vny) * T(0.5);
        T vbr = (vr + vnx) * T(0.5);
        T vbz = (vz + vnz) * T(0.5);
        T jmv = wq * vbt;
        acc_ind += (double)(jmv * Et);
        if (!a.implicit) acc_es += (double)(wq * (vbr * Er + vbz * Ez));
        add4(a.jm, NR, iz, ir, jmv * w00, jmv * w01, jmv * w10, jmv * w11);
        // move (cell units): r' = |(r + a, b)| written as r + delta
        T am = vnx * S.dtr, bm = vny * S.dtr, cm = vnz * S.dtz;
        T rho = (T)ir + dr;
        T x1 = rho + am;
        T rp = sqrt_t(x1 * x1 + bm * bm);
        T den = rho + rp;
        T delta = (den > T(0.0)) ? (am * (rho + x1) + bm * bm) / den : T(0.0);
        T vr2 = vnx, vt2 = vny;
        if (rp > T(0.0)) {
            T inv = one / rp;
            T ca = x1 * inv, sa = bm * inv;
            vr2 = ca * vnx + sa * vny;
            vt2 = ca * vny - sa * vnx;
        }
        T drn = dr + delta;
        T dzn = dz + cm;
        T kr = fmin_t(fmax_t(floor_t(drn), T(-1048576.0)), T(1048576.0));
        drn = drn - kr;
        int ir2 = ir + (int)kr;
        if (drn >= one) {
            drn = drn - one;
            ir2 += 1;
        }
        T kz = fmin_t(fmax_t(floor_t(dzn), T(-1048576.0)), T(1048576.0));
        dzn = dzn - kz;
        int iz2 = iz + (int)kz;
        if (dzn >= one) {
            dzn = dzn - one;
            iz2 += 1;
        }
        if (ir2 < 0) {
            ir2 = 0;
            drn = T(0.0);
        }
        // boundaries: electrode z < 0, wall r >= R, window z >= z_win
        bool he = iz2 < 0;
        bool hw = !he && ir2 >= nr;
        bool hd = !he && !hw && iz2 >= a.i_win;
        bool emit = false;
        if (sp == 1 && S.see_g > T(0.0) && (he || hw || hd))
            emit = see_emit(cc, step, S, P.uid[q], he ? 0 : (hw ? 1 : 2), (uint32_t)(iz * nr + ir), dr, dz, wrel);
        if (hd) {
            const T qd = emit ? wq * T(2.0) : wq;
            T rpos = (T)ir2 + drn;
            int j0 = (int)floor_t(rpos);
            T fr = rpos - (T)j0;
            atomicAdd(&a.win[a.i_win * NR + j0], (double)(qd * (one - fr)));
            atomicAdd(&a.win[a.i_win * NR + min(j0 + 1, nr)], (double)(qd * fr));
        }
        const bool alive = !(he || hw || hd);
        uint32_t ncell = kDead;
        if (alive) {
            ncell = (uint32_t)(iz2 * nr + ir2);
            T wa2 = one - drn, wb2 = one - dzn;
            add4(a.rho[sp], NR, iz2, ir2, wq * (wa2 * wb2), wq * (drn * wb2), wq * (wa2 * dzn),
                 wq * (drn * dzn));
            uint32_t r = philox2x32_10(P.uid[q], (step & 0x7FFFFFFFu) | ((uint32_t)sp << 31), a.key0 ^ a.key1);
            if (T(u01(r)) < S.pnull) {
                if (sp == 0)
                    electron_collision(cc, step, S, P.uid[q], vr2, vt2, vnz, ncell, drn, dzn, cnt, wrel);
                else
                    ion_collision(cc, step, S, P.uid[q], vr2, vt2, vnz, cnt);
            }
        } else {
            ++cnt[7 + sp];
        }
        P.cell[q] = ncell;
        P.dr[q] = alive ? drn : T(0.0);
        P.dz[q] = alive ? dzn : T(0.0);
        P.vr[q] = vr2;
        P.vt[q] = vt2;
        P.vz[q] = vnz;
    }
    // block reduction of the tallies
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        acc_ind += __shfl_xor_sync(0xffffffffu, acc_ind, o);
        acc_es += __shfl_xor_sync(0xffffffffu, acc_es, o);
    }
    for (int k = 0; k < 10; ++k) cnt[k] = __reduce_add_sync(0xffffffffu, cnt[k]);
    if (lane == 0) {
        s_f[warp][0] = acc_ind;
        s_f[warp][1] = acc_es;
        for (int k = 0; k < 10; ++k) s_c[warp][k] = cnt[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double si = 0, se = 0;
        unsigned long long tot[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
            si += s_f[w][0];
            se += s_f[w][1];
            for (int k = 0; k < 10; ++k) tot[k] += s_c[w][k];
        }
        DevState* st = a.st;
        atomicAdd(&st->p_ind_step, si);
        atomicAdd(&st->p_es_step, se);
        const int map[7] = {C_E_EL, C_E_EX, C_E_IZ, C_I_CX, C_I_ISO, C_NUVIOL, C_PSTEPS};
        for (int k = 0; k < 7; ++k)
            if (tot[k]) {
                atomicAdd(&st->cnt[map[k]], tot[k]);
                atomicAdd(&st->per[map[k]], tot[k]);
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

void launch_push_plain(Cell* c, cudaStream_t st) {
    PlainArgs<double> a;
    for (int s = 0; s < 2; ++s) {
        a.p[s] = c->pd[s][c->cur[s]];
        a.sp[s] = c->scd[s];
    }
    a.nslot = c->d_nslot;
    a.F = c->d_F64;
    a.rho[0] = c->d_rho64;
    a.rho[1] = c->d_rho64 + c->nnodes;
    a.implicit = c->implicit ? 1 : 0;
    a.jm = c->d_jm64;
    a.win = c->d_win;
    a.nr = c->nr;
    a.NR = c->NR;
    a.i_win = c->i_win;
    a.step = &c->d_st->step;
    a.key0 = (uint32_t)(c->cfg.seed & 0xffffffffu);
    a.key1 = (uint32_t)(c->cfg.seed >> 32);
    a.ev = c->d_events64;
    a.ev_cap = c->event_cap;
    a.st = c->d_st;
    // grid: a whole number of waves of 8 blocks per SM over the slots of both species
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t slots = c->cap[0] + c->cap[1];
    int64_t want = (slots + 255) / 256;
    int64_t blocks = (int64_t)nsm * 8;
    if (want < blocks) blocks = want < 1 ? 1 : want;
    push_plain<double><<<(unsigned)blocks, 256, 0, st>>>(a);
    count_launch();
}

}  // namespace pp
