// Stochastic weighted split-merge particle control (the GEC-type runs of
// Sec. 3.4 keep the macroparticle count of every cell near a target with an
// inherited split-merge module that the paper does not define; the reading
// implemented here is stated with pp_config.sm_every).
//
// One pass over a species, after the step's append:
//   sm_count    live particles per cell;
//   sm_plan     one block: which cells act (merge above sm_max, split below
//               sm_min, cells above kSmCap left alone), the exclusive scans
//               that place each acting cell's particles in `perm` and its new
//               copies after the store's used slots, the list of acting cells,
//               and whether the copies fit the store;
//   sm_scatter  the slots of the acting cells' particles, grouped by cell;
//   sm_apply    one block per acting cell: the cell's particles sorted by uid
//               in shared memory (bitonic), then its merges or splits;
//   sm_finish   slot count, uids, live count and counters.
// Merges keep one member of each pair (its slot, uid and state) with the
// summed weight and mark the other slot dead (the next counting sort drops
// it); splits halve a weight and write a copy with a new uid.
#include "pp_internal.h"
#include "pp_mcc.cuh"

namespace pp {

constexpr int kSmCap = 4096;             // particles of one cell the pass handles
constexpr int kSmThreads = 256;
constexpr int kSmPlanThreads = 1024;

__device__ __forceinline__ bool sm_acts(uint32_t n, int nmin, int nmax) {
    return n > (uint32_t)nmax || (n > 0u && n < (uint32_t)nmin);
}

__global__ void sm_count(const uint32_t* cell, const int* nslot, int sp, uint32_t* cnt) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nslot[sp]) return;
    const uint32_t c = cell[idx];
    if (c != kDead) atomicAdd(&cnt[c], 1u);
}

// exclusive block scan of one value per thread; returns the thread's offset,
// *total gets the sum
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* buf, uint32_t* total) {
    const int t = threadIdx.x;
    buf[t] = v;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const uint32_t x = t >= o ? buf[t - o] : 0u;
        __syncthreads();
        buf[t] += x;
        __syncthreads();
    }
    const uint32_t incl = buf[t];
    *total = buf[blockDim.x - 1];
    __syncthreads();
    return incl - v;
}

__global__ void __launch_bounds__(kSmPlanThreads) sm_plan(const uint32_t* cnt, int ncell, int target, int nmin,
                                                          int nmax, uint32_t* start, uint32_t* cursor,
                                                          uint32_t* soff, int* list, const int* nslot, int sp,
                                                          int64_t cap, DevState* st) {
    __shared__ uint32_t buf[kSmPlanThreads];
    const int t = threadIdx.x;
    const int per = (ncell + kSmPlanThreads - 1) / kSmPlanThreads;
    const int lo = min(t * per, ncell), hi = min(lo + per, ncell);
    uint32_t sn = 0, ss = 0, sa = 0, sk = 0;
    for (int c = lo; c < hi; ++c) {
        const uint32_t n = cnt[c];
        if (!sm_acts(n, nmin, nmax)) continue;
        if (n > (uint32_t)kSmCap) {
            ++sk;
            continue;
        }
        sn += n;
        ++sa;
        if (n < (uint32_t)nmin) ss += min((uint32_t)target - n, n);
    }
    uint32_t tn, ts, ta, tk;
    uint32_t on = block_excl_scan(sn, buf, &tn);
    uint32_t os = block_excl_scan(ss, buf, &ts);
    uint32_t oa = block_excl_scan(sa, buf, &ta);
    block_excl_scan(sk, buf, &tk);
    for (int c = lo; c < hi; ++c) {
        const uint32_t n = cnt[c];
        if (!sm_acts(n, nmin, nmax) || n > (uint32_t)kSmCap) continue;
        start[c] = on;
        cursor[c] = on;
        soff[c] = os;
        list[oa] = c;
        on += n;
        ++oa;
        if (n < (uint32_t)nmin) os += min((uint32_t)target - n, n);
    }
    if (t == 0) {
        st->sm_nlist = (int)ta;
        st->sm_split_total = (int)ts;
        const bool fits = (int64_t)nslot[sp] + (int64_t)ts <= cap;
        st->sm_split_ok = fits ? 1 : 0;
        if (!fits) st->status |= PP_ST_CAPACITY;
        st->ctl[3] += (unsigned long long)tk;
    }
}

__global__ void sm_scatter(const uint32_t* cell, const int* nslot, int sp, const uint32_t* cnt, int nmin, int nmax,
                           uint32_t* cursor, uint32_t* perm) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nslot[sp]) return;
    const uint32_t c = cell[idx];
    if (c == kDead) return;
    const uint32_t n = cnt[c];
    if (!sm_acts(n, nmin, nmax) || n > (uint32_t)kSmCap) return;
    perm[atomicAdd(&cursor[c], 1u)] = (uint32_t)idx;
}

template <typename T>
__global__ void __launch_bounds__(kSmThreads) sm_apply(PBuf<T> P, const int* nslot, int sp, const uint32_t* cnt,
                                                       const uint32_t* start, const uint32_t* soff,
                                                       const int* list, const uint32_t* perm,
                                                       const uint32_t* next_uid, int target, int nmin, int nmax,
                                                       const unsigned long long* step_ctr, uint32_t key0,
                                                       uint32_t key1, DevState* st) {
    __shared__ unsigned long long key[kSmCap];      // (uid << 32) | slot
    __shared__ unsigned s_merged;
    const uint32_t step = (uint32_t)(*step_ctr);
    const int nlist = st->sm_nlist;
    const bool split_ok = st->sm_split_ok != 0;
    const int base_slot = nslot[sp];
    const uint32_t base_uid = next_uid[sp];
    if (threadIdx.x == 0) s_merged = 0u;
    for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
        const int c = list[li];
        const int n = (int)cnt[c];
        const uint32_t s0 = start[c];
        int npow = 1;
        while (npow < n) npow <<= 1;
        __syncthreads();
        for (int j = threadIdx.x; j < npow; j += kSmThreads) {
            if (j < n) {
                const uint32_t slot = perm[s0 + j];
                key[j] = ((unsigned long long)P.uid[slot] << 32) | slot;
            } else {
                key[j] = ~0ull;
            }
        }
        __syncthreads();
        for (int k = 2; k <= npow; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < npow; i += kSmThreads) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const unsigned long long x = key[i], y = key[ixj];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) {
                            key[i] = y;
                            key[ixj] = x;
                        }
                    }
                }
                __syncthreads();
            }
        if (n > nmax) {
            const int k = min(n - target, n / 2);
            for (int j = threadIdx.x; j < k; j += kSmThreads) {
                const uint32_t a = (uint32_t)key[2 * j], b = (uint32_t)key[2 * j + 1];
                const T wa = P.w[a], wb = P.w[b];
                const T ws = wa + wb;
                const U4 u = draw4(P.uid[a], step, 5u, (uint32_t)sp, key0, key1);
                const bool keep_a = T(u.a) * ws < wa;
                const uint32_t surv = keep_a ? a : b, gone = keep_a ? b : a;
                P.w[surv] = ws;
                P.cell[gone] = kDead;
                P.dr[gone] = T(0.0);
                P.dz[gone] = T(0.0);
            }
            if (threadIdx.x == 0) s_merged += (unsigned)k;
        } else if (split_ok) {
            const int k = min(target - n, n);
            const uint32_t o = soff[c];
            for (int j = threadIdx.x; j < k; j += kSmThreads) {
                const uint32_t a = (uint32_t)key[j];
                const T wh = P.w[a] * T(0.5);
                P.w[a] = wh;
                const int d = base_slot + (int)(o + (uint32_t)j);
                P.cell[d] = P.cell[a];
                P.dr[d] = P.dr[a];
                P.dz[d] = P.dz[a];
                P.vr[d] = P.vr[a];
                P.vt[d] = P.vt[a];
                P.vz[d] = P.vz[a];
                P.uid[d] = base_uid + o + (uint32_t)j;
                P.w[d] = wh;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_merged) {
        atomicAdd(&st->live[sp], (unsigned long long)(-(long long)s_merged));
        atomicAdd(&st->ctl[2], (unsigned long long)s_merged);
    }
}

// slot count, uids, live count and split counter; the per-cell counts are
// cleared for the next pass
__global__ void sm_finish(int* nslot, uint32_t* next_uid, int sp, uint32_t* cnt, int ncell, DevState* st) {
    __shared__ int s_total;
    if (threadIdx.x == 0) {
        const int total = st->sm_split_ok ? st->sm_split_total : 0;
        s_total = total;
        nslot[sp] += total;
        next_uid[sp] += (uint32_t)total;
        st->live[sp] += (unsigned long long)total;
        st->ctl[1] += (unsigned long long)total;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < ncell + 2; q += blockDim.x) cnt[q] = 0u;
}

template <typename T>
static void split_merge_species(Cell* c, PBuf<T> P, int sp, cudaStream_t st) {
    const int ncell = c->i_win * c->nr;
    const unsigned nb = (unsigned)((c->cap[sp] + 255) / 256);
    sm_count<<<nb, 256, 0, st>>>(P.cell, c->d_nslot, sp, c->d_sm_cnt);
    sm_plan<<<1, kSmPlanThreads, 0, st>>>(c->d_sm_cnt, ncell, c->sm_target, c->sm_min, c->sm_max, c->d_sm_start,
                                          c->d_sm_cursor, c->d_sm_soff, c->d_sm_list, c->d_nslot, sp, c->cap[sp],
                                          c->d_st);
    sm_scatter<<<nb, 256, 0, st>>>(P.cell, c->d_nslot, sp, c->d_sm_cnt, c->sm_min, c->sm_max, c->d_sm_cursor,
                                   c->d_sm_perm);
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::min<long long>((long long)nsm * 4, std::max(ncell, 1));
    sm_apply<T><<<grid, kSmThreads, 0, st>>>(P, c->d_nslot, sp, c->d_sm_cnt, c->d_sm_start, c->d_sm_soff,
                                             c->d_sm_list, c->d_sm_perm, c->d_next_uid, c->sm_target, c->sm_min,
                                             c->sm_max, &c->d_st->step, (uint32_t)(c->cfg.seed & 0xffffffffu),
                                             (uint32_t)(c->cfg.seed >> 32), c->d_st);
    sm_finish<<<1, kSmPlanThreads, 0, st>>>(c->d_nslot, c->d_next_uid, sp, c->d_sm_cnt, ncell, c->d_st);
    count_launch(5);
}

void launch_split_merge(Cell* c, cudaStream_t st) {
    for (int sp = 0; sp < 2; ++sp) {
        if (c->fp64)
            split_merge_species<double>(c, c->pd[sp][c->cur[sp]], sp, st);
        else
            split_merge_species<float>(c, c->pb[sp][c->cur[sp]], sp, st);
    }
}

}  // namespace pp
