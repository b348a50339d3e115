// Counter-based random numbers and the null-collision Monte Carlo kinematics
// shared by the particle kernels, written over the state type T (float for
// the fused kernel, double for the plain FP64 form).  Arithmetic is plain IEEE
// in T with no contraction (the library is built with --fmad=false), in the
// operation order of the oracle's instantiation of the same type.
#pragma once

#include "pp_internal.h"

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

// Philox2x32-10 (same paper): round (c0, c1; k) -> (hi(M c0) ^ k ^ c1, lo(M c0)),
// M = 0xD256D193, key bumped by 0x9E3779B9; first output only
__device__ __forceinline__ uint32_t philox2x32_10(uint32_t c0, uint32_t c1, uint32_t k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) k += 0x9E3779B9u;
        uint32_t hi = __umulhi(0xD256D193u, c0), lo = 0xD256D193u * c0;
        c0 = hi ^ k ^ c1;
        c1 = lo;
    }
    return c0;
}

// ((x >> 9) + 0.5) * 2^-23, exact in float32 (and in double), in (0, 1)
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

// ---------------------------------------------------------------- math of either type
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }
__device__ __forceinline__ float log_t(float x) { return logf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }
__device__ __forceinline__ float fmax_t(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double fmax_t(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float fmin_t(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double fmin_t(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float floor_t(float x) { return floorf(x); }
__device__ __forceinline__ double floor_t(double x) { return floor(x); }
__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

// ---------------------------------------------------------------- cross sections
// electron-Ar (units 1e-20 m^2) at energy x (eV); project-defined rational fits
template <typename T>
__device__ __forceinline__ void sigma_e(T x, T& el, T& ex, T& iz) {
    const T e_exc = T(11.55), e_ion = T(15.76);
    T y = x - T(0.23);
    T y2 = y * y;
    el = (T(0.1) + T(14.0) * y2 / (y2 + T(4.0))) / (T(1.0) + x / T(50.0));
    T ye = x - e_exc;
    ex = (x > e_exc) ? T(1.2) * ye / (ye * ye / T(30.0) + ye + T(8.0)) : T(0.0);
    T yi = x - e_ion;
    iz = (x > e_ion) ? T(3.0) * yi / (yi * yi / T(60.0) + yi + T(30.0)) : T(0.0);
}

// Ar+-Ar charge exchange and isotropic elastic (units 1e-19 m^2) at lab energy x
template <typename T>
__device__ __forceinline__ void sigma_i(T x, T& cx, T& iso) {
    T sq = sqrt_t(x);
    cx = T(2.0) + T(3.0) / (T(1.0) + sq);
    iso = T(1.0) + T(2.0) / (T(1.0) + sq);
}

template <typename T>
__device__ __forceinline__ void iso_dir(T u2, T u3, T& dx, T& dy, T& dz) {
    T c = T(1.0) - T(2.0) * u2;
    T s = sqrt_t(fmax_t(T(1.0) - c * c, T(0.0)));
    T sp, cp;
    sincospi_t(T(2.0) * u3, &sp, &cp);
    dx = s * cp;
    dy = s * sp;
    dz = c;
}

template <typename T>
__device__ __forceinline__ void gauss3(T a, T b, T c, T d, T& n0, T& n1, T& n2) {
    T ra = sqrt_t(T(-2.0) * log_t(a));
    T rc = sqrt_t(T(-2.0) * log_t(c));
    T sb, cb, sd, cd;
    sincospi_t(T(2.0) * b, &sb, &cb);
    sincospi_t(T(2.0) * d, &sd, &cd);
    n0 = ra * cb;
    n1 = ra * sb;
    n2 = rc * cd;
}

// ---------------------------------------------------------------- collisions
// What a collision needs besides the particle: RNG key, the ionisation event
// buffer, device state (event count, status) and the ion gas thermal speed.
template <typename T>
struct CollCtx {
    uint32_t key0, key1;
    EventT<T>* ev;
    int ev_cap;
    DevState* st;
    T vth_gas_ion;
};

// e-Ar: process choice r = u1 nu_max against the cumulative frequencies,
// isotropic lab-frame scattering, elastic loss 2m/M (1 - cos chi), excitation
// threshold, ionisation with the excess energy split equally and an Ar+ drawn
// from the gas Maxwellian (recorded as an event, appended after the push).
// cnt: 0 elastic, 1 excitation, 2 ionisation, 5 nu_max violations.
template <typename T>
__device__ __forceinline__ void electron_collision(const CollCtx<T>& a, uint32_t step, const SpecT<T>& S,
                                                   uint32_t uid, T& vx, T& vy, T& vz, uint32_t cell, T drn,
                                                   T dzn, unsigned* cnt, T w = T(1.0)) {
    U4 u = draw4(uid, step, 0u, 0u, a.key0, a.key1);
    T x = vx, y = vy, z = vz;
    T v2 = x * x + y * y + z * z;
    T g = sqrt_t(v2);
    T en = v2 * S.ce;
    T s_el, s_ex, s_iz;
    sigma_e(en, s_el, s_ex, s_iz);
    T nu_el = S.ng * s_el * g;
    T nu_ex = S.ng * s_ex * g;
    T nu_iz = S.ng * s_iz * g;
    T r = T(u.b) * S.numax;
    T c1 = nu_el, c2 = c1 + nu_ex, c3 = c2 + nu_iz;
    if (c3 > S.numax) ++cnt[5];
    int proc = (r < c1) ? 0 : (r < c2) ? 1 : (r < c3) ? 2 : 3;
    if (proc == 3) return;
    const T one = T(1.0);
    T dx, dy, dzz;
    iso_dir(T(u.c), T(u.d), dx, dy, dzz);
    T gn;
    if (proc == 0) {
        T cosx = (g > T(0.0)) ? (x * dx + y * dy + z * dzz) / g : T(0.0);
        gn = g * sqrt_t(one - S.loss * (one - cosx));
        ++cnt[0];
    } else if (proc == 1) {
        gn = sqrt_t(fmax_t(en - T(11.55), T(0.0)) * S.inv_ce);
        ++cnt[1];
    } else {
        T eh = fmax_t(en - T(15.76), T(0.0)) * T(0.5);
        gn = sqrt_t(eh * S.inv_ce);
        ++cnt[2];
        U4 a1 = draw4(uid, step, 1u, 0u, a.key0, a.key1);
        U4 b1 = draw4(uid, step, 2u, 0u, a.key0, a.key1);
        T ex_, ey_, ez_, g0, g1, g2;
        iso_dir(T(a1.a), T(a1.b), ex_, ey_, ez_);
        gauss3(T(a1.c), T(a1.d), T(b1.a), T(b1.b), g0, g1, g2);
        int slot = atomicAdd(&a.st->n_events, 1);
        if (slot < a.ev_cap) {
            EventT<T> e;
            e.parent = uid;
            e.cell = cell;
            e.dr = drn;
            e.dz = dzn;
            e.ve[0] = gn * ex_;
            e.ve[1] = gn * ey_;
            e.ve[2] = gn * ez_;
            e.vi[0] = a.vth_gas_ion * g0;
            e.vi[1] = a.vth_gas_ion * g1;
            e.vi[2] = a.vth_gas_ion * g2;
            e.w = w;
            e.kind = 0u;
            a.ev[slot] = e;
        } else {
            atomicOr(&a.st->status, (unsigned)PP_ST_EVENTS);
        }
    }
    vx = gn * dx;
    vy = gn * dy;
    vz = gn * dzz;
}

// Ion-induced secondary emission of an Ar+ absorbed on a surface (0
// electrode, 1 side wall, 2 window): with probability see_g (first uniform of
// draw call 3) one electron starts at the ion's last position inside the
// plasma (cell, dr, dz) with the ion's weight, its normal speed Rayleigh,
// v_s sqrt(-2 ln u_b), into the plasma, its tangential components
// v_s sqrt(-2 ln u_c) (cos, sin)(2 pi u_d).  Recorded as a kind-1 event.
// Returns whether the ion emitted.
template <typename T>
__device__ __forceinline__ bool see_emit(const CollCtx<T>& a, uint32_t step, const SpecT<T>& S, uint32_t uid,
                                         int surface, uint32_t cell, T dr, T dz, T w) {
    U4 u = draw4(uid, step, 3u, 1u, a.key0, a.key1);
    if (!(T(u.a) < S.see_g)) return false;
    const T rn = sqrt_t(T(-2.0) * log_t(T(u.b)));
    const T rt = sqrt_t(T(-2.0) * log_t(T(u.c)));
    T sd, cd;
    sincospi_t(T(2.0) * T(u.d), &sd, &cd);
    const T vn = S.see_vs * rn;
    const T t1 = S.see_vs * (rt * cd), t2 = S.see_vs * (rt * sd);
    EventT<T> e;
    e.parent = uid;
    e.cell = cell;
    e.dr = dr;
    e.dz = dz;
    if (surface == 0) {
        e.ve[0] = t1;
        e.ve[1] = t2;
        e.ve[2] = vn;
    } else if (surface == 1) {
        e.ve[0] = -vn;
        e.ve[1] = t1;
        e.ve[2] = t2;
    } else {
        e.ve[0] = t1;
        e.ve[1] = t2;
        e.ve[2] = -vn;
    }
    e.vi[0] = e.vi[1] = e.vi[2] = T(0.0);
    e.w = w;
    e.kind = 1u;
    int slot = atomicAdd(&a.st->n_events, 1);
    if (slot < a.ev_cap) {
        a.ev[slot] = e;
        atomicAdd(&a.st->n_see, 1);
    } else {
        atomicOr(&a.st->status, (unsigned)PP_ST_EVENTS);
    }
    return true;
}

// Ar+-Ar against a gas partner drawn from the 300 K Maxwellian: charge
// exchange takes the partner's velocity, isotropic elastic scatters in the
// centre-of-mass frame.  cnt: 3 cx, 4 isotropic, 5 nu_max violations.
template <typename T>
__device__ __forceinline__ void ion_collision(const CollCtx<T>& a, uint32_t step, const SpecT<T>& S, uint32_t uid,
                                              T& vx, T& vy, T& vz, unsigned* cnt) {
    U4 u = draw4(uid, step, 0u, 1u, a.key0, a.key1);
    U4 a1 = draw4(uid, step, 1u, 1u, a.key0, a.key1);
    T g0, g1, g2;
    gauss3(T(a1.a), T(a1.b), T(a1.c), T(a1.d), g0, g1, g2);
    T vnxn = S.vth_gas * g0, vnyn = S.vth_gas * g1, vnzn = S.vth_gas * g2;
    T x = vx, y = vy, z = vz;
    T gx = x - vnxn, gy = y - vnyn, gz = z - vnzn;
    T g2s = gx * gx + gy * gy + gz * gz;
    T g = sqrt_t(g2s);
    T en = g2s * S.ce;
    T s_cx, s_iso;
    sigma_i(en, s_cx, s_iso);
    T nu_cx = S.ng * s_cx * g;
    T nu_iso = S.ng * s_iso * g;
    T r = T(u.b) * S.numax;
    T c1 = nu_cx, c2 = c1 + nu_iso;
    if (c2 > S.numax) ++cnt[5];
    if (r < c1) {
        vx = vnxn;
        vy = vnyn;
        vz = vnzn;
        ++cnt[3];
    } else if (r < c2) {
        T dx, dy, dzz;
        iso_dir(T(u.c), T(u.d), dx, dy, dzz);
        T hg = g * T(0.5);
        vx = (x + vnxn) * T(0.5) + hg * dx;
        vy = (y + vnyn) * T(0.5) + hg * dy;
        vz = (z + vnzn) * T(0.5) + hg * dzz;
        ++cnt[4];
    }
}

}  // namespace pp
