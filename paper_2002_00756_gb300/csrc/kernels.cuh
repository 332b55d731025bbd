// Device kernels of the column multigrid solver (sm_103a).
//
// Layout: cell fields are level-major f[k * ncol + col], so the threads of a warp, one
// column each, read consecutive words at every level k.  Coefficients are stored in
// face form (see mesh.h): Th[k][face] for horizontal faces, Tv[kf][col] for vertical
// faces, with 1/area per column and 1/dz per level supplying the volume normalisation.
//
// All stencil kernels run one thread per vertical column and walk the column bottom to
// top, keeping the cells below / at / above k in registers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_pipeline.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace mg {

template <typename T, typename C>
struct Lvl {
    int n, ncol, nlev;
    const int32_t* nbr;   // [4][ncol]
    const int32_t* fof;   // [4][ncol]
    const C* Th;          // [nlev][2 ncol]
    const C* Tv;          // [nlev+1][ncol], rows 0 and nlev are zero
    const T* rA;          // [ncol] 1 / area
    const T* rdz;         // [nlev] 1 / dz
};

template <typename T, typename C>
__device__ __forceinline__ T ldc(const C* p) {
    return (T)__ldg(p);
}
template <>
__device__ __forceinline__ float ldc<float, __nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
}

template <typename T, typename X>
__device__ __forceinline__ T ldx(const X* p) {
    return (T)__ldg(p);
}

__device__ __forceinline__ int parent_col(int col, int n) {
    const int nn = n * n, p = col / nn, r = col - p * nn, j = r / n, i = r - j * n, nc = n >> 1;
    return p * nc * nc + (j >> 1) * nc + (i >> 1);
}

__device__ __forceinline__ int child_col_dev(int n_fine, int C, int q) {
    const int nc = n_fine >> 1, ncc = nc * nc;
    const int p = C / ncc, r = C - p * ncc, J = r / nc, I = r - J * nc;
    return p * n_fine * n_fine + (2 * J + (q >> 1)) * n_fine + 2 * I + (q & 1);
}

// Source of the current iterate x on the fine level of a kernel:
//   XM_PLAIN    x[k][col]
//   XM_ZERO     0 (the first sweep of a level)
//   XM_PROLONG  x[k][col] + xc[k][parent(col)]   (prolongation fused into the sweep)
//   XM_PROLONG0 xc[k][parent(col)]               (prolongation onto a zero iterate)
enum { XM_PLAIN = 0, XM_ZERO = 1, XM_PROLONG = 2, XM_PROLONG0 = 3 };

template <int MODE, typename T, typename X>
__device__ __forceinline__ T xval(const X* __restrict__ x, const T* __restrict__ xc, size_t o,
                                  size_t oc, int col, int par) {
    if (MODE == XM_ZERO) return T(0);
    T v = (MODE == XM_PROLONG0) ? T(0) : ldx<T>(x + o + col);
    if (MODE == XM_PROLONG || MODE == XM_PROLONG0) v += __ldg(xc + oc + par);
    return v;
}

// ---------------------------------------------------------------------------------------
// y = H x (Eq. helmholtz_operator): one thread per column, levels [k0, k0 + kchunk).
template <typename T, typename C, typename X, typename Y>
__global__ void __launch_bounds__(256) k_apply(Lvl<T, C> L, const X* __restrict__ x,
                                               Y* __restrict__ y, int kchunk) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.ncol) return;
    const size_t ncol = L.ncol, nf = 2 * ncol;
    const int k0 = blockIdx.y * kchunk;
    const int k1 = min(L.nlev, k0 + kchunk);
    int nb[4], fo[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        nb[s] = __ldg(L.nbr + s * ncol + c);
        fo[s] = __ldg(L.fof + s * ncol + c);
    }
    const T rA = __ldg(L.rA + c);
    T xm = k0 > 0 ? ldx<T>(x + (size_t)(k0 - 1) * ncol + c) : T(0);
    T x0 = ldx<T>(x + (size_t)k0 * ncol + c);
    T tdn = ldc<T>(L.Tv + (size_t)k0 * ncol + c);
    for (int k = k0; k < k1; ++k) {
        const size_t o = (size_t)k * ncol;
        const T xp = (k + 1 < L.nlev) ? ldx<T>(x + o + ncol + c) : T(0);
        const T tup = ldc<T>(L.Tv + o + ncol + c);
        const C* th = L.Th + (size_t)k * nf;
        T h = ldc<T>(th + fo[0]) * (x0 - ldx<T>(x + o + nb[0]));
        h += ldc<T>(th + fo[1]) * (x0 - ldx<T>(x + o + nb[1]));
        h += ldc<T>(th + fo[2]) * (x0 - ldx<T>(x + o + nb[2]));
        h += ldc<T>(th + fo[3]) * (x0 - ldx<T>(x + o + nb[3]));
        const T v = __ldg(L.rdz + k) * (tup * (x0 - xp) + tdn * (x0 - xm));
        y[o + c] = (Y)(x0 + (rA * h + v));
        xm = x0;
        x0 = xp;
        tdn = tup;
    }
}

// ---------------------------------------------------------------------------------------
// One block-Jacobi sweep (Eq. jacobi): x_out = x + omega Hz^{-1} (b - H x).
//
// Two threads per column solve its tridiagonal system from both ends (a twisted
// factorisation): the first half of a block's warps take the lower halves of its columns
// (32 consecutive columns per warp) and eliminate upwards from the surface, the second
// half take the upper halves of the same columns and eliminate downwards from the lid, so
// every copy and load of a warp touches one level.  With the coupling to the already-eliminated
// neighbour a_prev and to the next one a_next, every step is
//     m = a_prev / p_prev,  q = s + m q_prev,  p = q + a_next,  y = r + m y_prev
// (s = 1 + horizontal coefficients: pivots are sums of positive terms).  The two halves
// meet at rows h-1 and h; their 2x2 system
//     [p_A  -a_A] [d_A]   [y_A]
//     [-a_B  p_B] [d_B] = [y_B],   det = q_A p_B + a_A q_B  (no cancellation)
// is solved by both threads after an exchange through shared memory, then each half back-substitutes towards its
// end: d_i = y_i/p_i + e_i d_{i+1}, e_i = a_next/p_i, out_i = x_i + omega d_i.  The back
// substitution runs directly on the output,
//     out_i = w_i + e_i out_{i+1},   w_i = x_i + omega y_i/p_i - e_i x_{i+1},
// so the forward pass stashes (w_i, e_i) in shared memory and the iterate is never read
// again.  Compared with one thread per column this doubles the resident warps for the
// same stash and halves the serial recurrence.
//
// Latency hiding: the streams first met in DRAM (the next iterate of the own column, b,
// the E and N faces and the vertical face ahead) are copied DEEP steps ahead into a
// per-thread shared-memory ring with asynchronous copies (cp.async via the CUDA pipeline
// primitives), so they occupy no registers while in flight.  The lanes of a warp hold
// consecutive columns at the same level, so the E and W neighbour iterates are the
// adjacent lanes' own values (warp shuffles) and the W face is the left lane's staged E face
// (shared memory); only where a neighbour is not the adjacent column (ends of the lane
// group, panel edges) is it loaded.  Those loads, the N and S neighbours, the S face and the
// prolongation terms run SHAL steps ahead in a register ring; 1/dz comes from a per-block
// shared table.  Both rings are indexed statically: the step loop is unrolled by DEEP.
//
// Addressing: every array the walk touches is reached through a per-thread base pointer
// (column, neighbour column or face index already added) plus one running 32-bit offset
// kc = k * ncol (cells; 2 kc for the faces, k * ncol_c for the coarse level), so each
// access costs one multiply-add of the address; the host guarantees 2 nlev ncol < 2^32.
// The steps of the walk that need no end-of-column checks (both halves still have DEEP
// steps to stage) run in a loop without them; the last few run with the checks.
template <typename T>
struct SweepShal {
    T xh[4], tw, ts, ch[4], cn;
    T te, tn, tv;   // coefficients narrower than 4 bytes (BF16) travel here instead
};

// (launched with at most MG_SWEEP_BLOCK threads; four resident blocks is what the shared
// memory of the large levels allows, so registers are capped to match)
#ifndef MG_SWEEP_BLOCK
#define MG_SWEEP_BLOCK 128
#endif
#ifndef MG_SWEEP_BF16_PAIRS
#define MG_SWEEP_BF16_PAIRS 1
#endif
// 1: the first half of a block's warps take the lower halves of its columns and the second
// half the upper halves (32 columns per warp, blocks of a multiple of 64 threads); 0: lanes
// 0-15 and 16-31 of every warp take the two halves of the same 16 columns
#ifndef MG_SWEEP_WARP_HALVES
#define MG_SWEEP_WARP_HALVES 1
#endif
// P is the type of the column elimination (pivots, eliminated right-hand side, multipliers and
// the interface solve); P = T everywhere but in the finest-level sweeps of MG_FP32_P64, which
// eliminate FP32 data with FP64 pivots.  The stash (w_i, e_i) and the back substitution stay in T.
template <typename T, typename C, int MODE, typename X, typename B, typename O, bool BCOPY, int DEEP, int SHAL,
          typename P>
__global__ void __launch_bounds__(MG_SWEEP_BLOCK, 4) k_sweep(Lvl<T, C> L, const X* __restrict__ x, const T* __restrict__ xc,
                        int ncol_c, const B* __restrict__ b, T* __restrict__ bcopy,
                        O* __restrict__ xo, T omega) {
    static_assert(DEEP % SHAL == 0, "ring lengths");
    static_assert(sizeof(X) == sizeof(T), "iterate type");
    static_assert(DEEP * (sizeof(B) + sizeof(T)) >= 3 * sizeof(P), "the interface exchange reuses the ring");
    // asynchronous copies move 4, 8 or 16 bytes: a BF16 coefficient travels in the aligned
    // 4-byte pair that holds it (its neighbour in memory rides along) and is picked out of
    // the pair in the ring
    constexpr bool PAIR = sizeof(C) == 2;
    constexpr bool ASYNC_C = sizeof(C) >= 4 || (PAIR && MG_SWEEP_BF16_PAIRS);
    typedef typename std::conditional<PAIR, uint32_t, C>::type CW;   // ring word of a coefficient
    constexpr bool PRO = (MODE == XM_PROLONG || MODE == XM_PROLONG0);
    constexpr bool RAW = (MODE == XM_PLAIN || MODE == XM_PROLONG);   // reads the fine iterate
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nlev = L.nlev, hsteps = (nlev + 1) >> 1;
    const int tid = threadIdx.x, bd = blockDim.x;
    // shared memory: [ring of DEEP slots of b (B), xn (T), te, tn, tv (C, when staged)]
    // [stash 2 x hsteps (T)] [1/dz, nlev (T)]
    B* rb = reinterpret_cast<B*>(smem_raw);
    T* rx = reinterpret_cast<T*>(rb + (size_t)DEEP * bd);
    CW* rte = reinterpret_cast<CW*>(rx + (size_t)DEEP * bd);
    CW* rtn = rte + (size_t)DEEP * bd;
    CW* rtv = rtn + (size_t)DEEP * bd;
    T* sc = reinterpret_cast<T*>(ASYNC_C ? (unsigned char*)(rtv + (size_t)DEEP * bd)
                                         : (unsigned char*)rte);
    T* se = sc + (size_t)hsteps * bd;
    T* srdz = se + (size_t)hsteps * bd;   // [nlev]
    for (int k = threadIdx.x; k < nlev; k += bd) srdz[k] = __ldg(L.rdz + k);
    __syncthreads();
    const int lane = threadIdx.x & 31;
#if MG_SWEEP_WARP_HALVES
    const int nwh = bd >> 6;                       // warps per half
    const bool upper = (threadIdx.x >> 5) >= nwh;
    const int c_raw = blockIdx.x * (bd >> 1) + ((threadIdx.x >> 5) - (upper ? nwh : 0)) * 32 + lane;
    const int g = lane, glast = 31;                // lanes holding consecutive columns
#else
    const bool upper = lane >= 16;
    const int c_raw = blockIdx.x * (bd >> 1) + (threadIdx.x >> 5) * 16 + (lane & 15);
    const int g = lane & 15, glast = 15;
#endif
    const bool active = c_raw < L.ncol;
    const int c = active ? c_raw : L.ncol - 1;
    const int nsteps = upper ? nlev - hsteps : hsteps;
    const int dir = upper ? -1 : 1;
    const int kfirst = upper ? nlev - 1 : 0;
    const unsigned ncol = L.ncol;
    // offsets of level kfirst and their change per step
    const unsigned kc0 = (unsigned)kfirst * ncol, kcc0 = (unsigned)kfirst * (unsigned)ncol_c;
    const unsigned dkc = upper ? 0u - ncol : ncol, dkcc = upper ? 0u - (unsigned)ncol_c : (unsigned)ncol_c;
    int nb[4], fo[4], pn[4] = {0, 0, 0, 0}, pc = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        nb[s] = __ldg(L.nbr + s * ncol + c);
        fo[s] = __ldg(L.fof + s * ncol + c);
    }
    if (PRO) {
        pc = parent_col(c, L.n);
#pragma unroll
        for (int s = 0; s < 4; ++s) pn[s] = parent_col(nb[s], L.n);
    }
    const T rA = __ldg(L.rA + c);
    // E / W neighbours that are the adjacent lanes of the group
    const bool shE = g != glast && nb[0] == c + 1;
    const bool shW = g != 0 && nb[1] == c - 1;
    // the W face is the left lane's E face when it is the same face
    const bool shWf = ASYNC_C && shW && fo[1] == __ldg(L.fof + (c > 0 ? c - 1 : 0));
    // per-thread bases; the face arrays advance by 2 kc, the vertical face towards the next
    // level of the walk is Tv[k+1] going up and Tv[k] going down
    const B* pb = b + c;
    const X* px = x + c;
    const X* pxh[4] = {x + nb[0], x + nb[1], x + nb[2], x + nb[3]};
    const C* pth[4] = {L.Th + fo[0], L.Th + fo[1], L.Th + fo[2], L.Th + fo[3]};
    const C* ptv = L.Tv + c + (upper ? 0u : ncol);
    const T* pch[4] = {xc + pn[0], xc + pn[1], xc + pn[2], xc + pn[3]};
    const T* pcc = xc + pc;
    // BF16 pairs: word bases (offsets in words: kc for the faces, whose level holds 2 ncol
    // values, kc / 2 for the vertical faces) and the half of the word that holds the value
    const uint32_t* pte2 = reinterpret_cast<const uint32_t*>(L.Th) + (fo[0] >> 1);
    const uint32_t* ptn2 = reinterpret_cast<const uint32_t*>(L.Th) + (fo[2] >> 1);
    const uint32_t* ptv2 = reinterpret_cast<const uint32_t*>(L.Tv) + ((c + (upper ? 0u : ncol)) >> 1);
    auto half = [](uint32_t w, int h) -> T { return (T)__uint_as_float(h ? (w & 0xffff0000u) : (w << 16)); };

    auto stage = [&](int i, int slot, unsigned kc, bool chk) {
        if (!chk || i < nsteps) {
            const int so = slot * bd + tid;
            __pipeline_memcpy_async(rb + so, pb + kc, sizeof(B));
            if (RAW) {
                const bool in = !chk || i + 1 < nsteps || (upper ? kfirst - i - 1 >= 0 : kfirst + i + 1 < nlev);
                __pipeline_memcpy_async(rx + so, px + (in ? kc + dkc : kc), sizeof(T), in ? 0 : sizeof(T));
            }
            if (ASYNC_C && PAIR) {
                __pipeline_memcpy_async(rte + so, pte2 + kc, 4);
                __pipeline_memcpy_async(rtn + so, ptn2 + kc, 4);
                __pipeline_memcpy_async(rtv + so, ptv2 + (kc >> 1), 4);
            } else if (ASYNC_C) {
                __pipeline_memcpy_async(rte + so, pth[0] + 2 * kc, sizeof(C));
                __pipeline_memcpy_async(rtn + so, pth[2] + 2 * kc, sizeof(C));
                __pipeline_memcpy_async(rtv + so, ptv + kc, sizeof(C));
            }
        }
        __pipeline_commit();
    };
    auto load_shal = [&](int i, unsigned kc, unsigned kcc, SweepShal<T>& d) {
        if (RAW) {
            if (!shE) d.xh[0] = ldx<T>(pxh[0] + kc);
            if (!shW) d.xh[1] = ldx<T>(pxh[1] + kc);
            d.xh[2] = ldx<T>(pxh[2] + kc);
            d.xh[3] = ldx<T>(pxh[3] + kc);
        }
        if (PRO) {
            if (!shE) d.ch[0] = __ldg(pch[0] + kcc);
            if (!shW) d.ch[1] = __ldg(pch[1] + kcc);
            d.ch[2] = __ldg(pch[2] + kcc);
            d.ch[3] = __ldg(pch[3] + kcc);
            const int k = kfirst + dir * i, kn = k + dir;
            d.cn = (kn >= 0 && kn < nlev) ? __ldg(pcc + (kcc + dkcc)) : T(0);   // offsets wrap mod 2^32: add them first
        }
        if (!shWf) d.tw = ldc<T>(pth[1] + 2 * kc);
        d.ts = ldc<T>(pth[3] + 2 * kc);
        if (!ASYNC_C) {
            d.te = ldc<T>(pth[0] + 2 * kc);
            d.tn = ldc<T>(pth[2] + 2 * kc);
            d.tv = ldc<T>(ptv + kc);
        }
    };

    unsigned kc_st = kc0;   // offset of the next level to stage
#pragma unroll
    for (int j = 0; j < DEEP; ++j) {
        stage(j, j, kc_st, true);
        kc_st += dkc;
    }
    SweepShal<T> sr[SHAL];
    unsigned kc_sh = kc0, kcc_sh = kcc0;   // offsets of the next level for the register ring
#pragma unroll
    for (int j = 0; j < SHAL; ++j) {
        if (j < nsteps) load_shal(j, kc_sh, kcc_sh, sr[j]);
        kc_sh += dkc;
        kcc_sh += dkcc;
    }
    T xprev = T(0), x0 = T(0), tprev = T(0);
    if (RAW) x0 = ldx<T>(px + kc0);
    if (PRO) x0 += __ldg(pcc + kcc0);
    P q = P(0), ip = P(0), y = P(0), anext = P(0);
    T* psc = sc + tid;
    T* pse = se + tid;
    const T* prdz = srdz + kfirst;

    auto step = [&](int i, int j, bool chk) {
        __pipeline_wait_prior(DEEP - 1);
        __syncwarp();   // every lane's copies of this slot are complete and visible
        const int so = j * bd + tid;
        const T bk = (T)rb[so];
        T xn = RAW ? rx[so] : T(0);
        T te = T(0), tn = T(0), tv = T(0), twl = T(0);
        if (ASYNC_C) {
            if constexpr (PAIR) {
                te = half(rte[so], fo[0] & 1);
                tn = half(rtn[so], fo[2] & 1);
                tv = half(rtv[so], c & 1);
                if (shWf) twl = half(rte[so - 1], fo[1] & 1);
            } else {
                te = (T)rte[so];
                tn = (T)rtn[so];
                tv = (T)rtv[so];
                if (shWf) twl = (T)rte[so - 1];
            }
        }
        __syncwarp();   // reads of the slot are done before it is refilled
        stage(i + DEEP, j, kc_st, chk);
        kc_st += dkc;
        // neighbour iterates at this level from the adjacent lanes (all lanes take part)
        const T xEl = __shfl_down_sync(0xffffffffu, x0, 1);
        const T xWl = __shfl_up_sync(0xffffffffu, x0, 1);
        if (!chk || i < nsteps) {
            const SweepShal<T> e = sr[j % SHAL];
            if (!ASYNC_C) {
                te = e.te;
                tn = e.tn;
                tv = e.tv;
            }
            if (!chk || i + SHAL < nsteps) load_shal(i + SHAL, kc_sh, kcc_sh, sr[j % SHAL]);
            if (PRO) xn += e.cn;
            T xh[4] = {T(0), T(0), T(0), T(0)};
            if (RAW) {
#pragma unroll
                for (int s = 0; s < 4; ++s) xh[s] = e.xh[s];
            }
            if (PRO) {
#pragma unroll
                for (int s = 0; s < 4; ++s) xh[s] += e.ch[s];
            }
            if (shE) xh[0] = xEl;
            if (shW) xh[1] = xWl;
            const T tw = shWf ? twl : e.tw;
            const T rdz = *prdz;
            if (BCOPY) bcopy[kc_sh - SHAL * dkc + c] = bk;
            T r = bk;
            if (MODE != XM_ZERO) {
                T hx = te * (x0 - xh[0]);
                hx += tw * (x0 - xh[1]);
                hx += tn * (x0 - xh[2]);
                hx += e.ts * (x0 - xh[3]);
                r -= x0 + (rA * hx + rdz * (tv * (x0 - xn) + tprev * (x0 - xprev)));
            }
            anext = P(rdz) * P(tv);
            const P m = (P(rdz) * P(tprev)) * ip;
            q = (P(1) + P(rA) * P((te + tw) + (tn + e.ts))) + m * q;
            const P p = q + anext;
            y = P(r) + m * y;
            ip = P(1) / p;
            const P ei = anext * ip;
            *psc = T(P(x0) + P(omega) * (y * ip) - ei * P(xn));
            *pse = T(ei);
            xprev = x0;
            x0 = xn;
            tprev = tv;
        }
        psc += bd;
        pse += bd;
        prdz += dir;
        kc_sh += dkc;
        kcc_sh += dkcc;
    };
    // steady state: every step of both halves stages DEEP ahead and loads SHAL ahead
    const int nfree = nlev - hsteps - DEEP;   // steps i < nfree need no checks in either half
    int i0 = 0;
    for (; i0 + DEEP <= nfree; i0 += DEEP) {
#pragma unroll
        for (int j = 0; j < DEEP; ++j) step(i0 + j, j, false);
    }
    for (; i0 < hsteps; i0 += DEEP) {
#pragma unroll
        for (int j = 0; j < DEEP; ++j) step(i0 + j, j, true);
    }
    __pipeline_wait_prior(0);
    // interface rows h-1 (lower half) and h (upper half)
#if MG_SWEEP_WARP_HALVES
    // through shared memory (the ring, free once every warp has left it) from the thread
    // tid ^ (bd / 2) that holds the other half of the column
    __syncthreads();
    P* xch = reinterpret_cast<P*>(smem_raw);
    xch[tid] = q;
    xch[bd + tid] = y;
    xch[2 * bd + tid] = anext;
    __syncthreads();
    const int pt = tid ^ (bd >> 1);
    const P qo = xch[pt], yo = xch[bd + pt], ao = xch[2 * bd + pt];
#else
    const P qo = __shfl_xor_sync(0xffffffffu, q, 16);
    const P yo = __shfl_xor_sync(0xffffffffu, y, 16);
    const P ao = __shfl_xor_sync(0xffffffffu, anext, 16);
#endif
    P dlt;
    if (nlev - hsteps == 0) {
        dlt = y * ip;   // a single level: nothing above, anext = 0
    } else {
        const P po = qo + ao;
        dlt = (y * po + anext * yo) / (q * po + anext * qo);
    }
    if (!active || nsteps == 0) return;
    // xprev holds the iterate at the last level of this half: out = x + omega d there
    T out = T(P(xprev) + P(omega) * dlt);
    O* po = xo + c;
    unsigned ko = kc0 + (unsigned)(nsteps - 1) * dkc;
    po[ko] = (O)out;
    if (nsteps < 2) return;
    const T* qsc = sc + (nsteps - 2) * bd + tid;
    const T* qse = se + (nsteps - 2) * bd + tid;
#pragma unroll 4
    for (int i = nsteps - 2; i >= 0; --i) {
        out = *qsc + *qse * out;
        ko -= dkc;
        po[ko] = (O)out;
        qsc -= bd;
        qse -= bd;
    }
}

// ---------------------------------------------------------------------------------------
// The same block-Jacobi sweep (same thread layout, same arithmetic in the same order, so the
// same result bit for bit) for FP32 levels of an even number NLEV of levels, with the
// elimination's stash (w_i, e_i) in registers instead of shared memory: every step of the
// walk is unrolled (NS = NLEV / 2 steps per half), so the stash is NS register pairs.  The
// shared memory the stash occupied holds instead a DEEP-slot ring that brings every value a
// step reads -- the own column's b, next iterate and E / N / vertical faces, and the N, S (and,
// at the ends of the lane group or across panel edges, E, W) neighbour iterates, the S and W
// faces and the prolongation terms -- by asynchronous 4-byte copies, so no step issues a
// global load: the walk waits only on its ring slot.
template <int NLEV>
struct SweepRsBlocks {   // resident blocks per SM: the stash of 70 levels needs the registers of 3
    static constexpr int value = NLEV > 50 ? 3 : 4;
};

template <int NLEV, int MODE, typename B, typename O, bool BCOPY, int DEEP>
__global__ void __launch_bounds__(MG_SWEEP_BLOCK, SweepRsBlocks<NLEV>::value)
    k_sweep_rs(Lvl<float, float> L, const float* __restrict__ x, const float* __restrict__ xc, int ncol_c,
               const B* __restrict__ b, float* __restrict__ bcopy, O* __restrict__ xo, float omega) {
    static_assert(NLEV % 2 == 0 && NLEV >= 2, "even level count");
    constexpr int NS = NLEV / 2;
    constexpr bool PRO = (MODE == XM_PROLONG || MODE == XM_PROLONG0);
    constexpr bool RAW = (MODE == XM_PLAIN || MODE == XM_PROLONG);
    constexpr bool BD = sizeof(B) == 8;
    // word slots of one ring entry (FP32): faces E, N, vertical ahead, S, W; iterates next, N, S,
    // E, W; prolongation terms next, N, S, E, W; b when it is FP32
    enum { W_TE, W_TN, W_TV, W_TS, W_TW, W_END0 };
    constexpr int W_XN = W_END0, W_XNB = W_XN + 1, W_XS = W_XN + 2, W_XE = W_XN + 3, W_XW = W_XN + 4;
    constexpr int W_END1 = RAW ? W_XN + 5 : W_END0;
    constexpr int W_CN = W_END1, W_CNB = W_CN + 1, W_CS = W_CN + 2, W_CE = W_CN + 3, W_CW = W_CN + 4;
    constexpr int W_END2 = PRO ? W_CN + 5 : W_END1;
    constexpr int W_B = W_END2;
    constexpr int NW = BD ? W_END2 : W_END2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, bd = blockDim.x;
    double* rbd = reinterpret_cast<double*>(smem_raw);                        // [DEEP][bd] (FP64 b)
    float* ring = reinterpret_cast<float*>(smem_raw + (BD ? (size_t)DEEP * bd * 8 : 0));   // [DEEP][NW][bd]
    float* srdz = ring + (size_t)DEEP * NW * bd;                              // [NLEV]
    for (int k = tid; k < NLEV; k += bd) srdz[k] = __ldg(L.rdz + k);
    __syncthreads();
    const int lane = tid & 31;
    const int nwh = bd >> 6;
    const bool upper = (tid >> 5) >= nwh;
    const int c_raw = blockIdx.x * (bd >> 1) + ((tid >> 5) - (upper ? nwh : 0)) * 32 + lane;
    const bool active = c_raw < L.ncol;
    const int c = active ? c_raw : L.ncol - 1;
    const int dir = upper ? -1 : 1;
    const int kfirst = upper ? NLEV - 1 : 0;
    const unsigned ncol = L.ncol;
    const unsigned kc0 = (unsigned)kfirst * ncol, kcc0 = (unsigned)kfirst * (unsigned)ncol_c;
    const unsigned dkc = upper ? 0u - ncol : ncol, dkcc = upper ? 0u - (unsigned)ncol_c : (unsigned)ncol_c;
    int nb[4], fo[4], pn[4] = {0, 0, 0, 0}, pc = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        nb[s] = __ldg(L.nbr + s * ncol + c);
        fo[s] = __ldg(L.fof + s * ncol + c);
    }
    if (PRO) {
        pc = parent_col(c, L.n);
#pragma unroll
        for (int s = 0; s < 4; ++s) pn[s] = parent_col(nb[s], L.n);
    }
    const float rA = __ldg(L.rA + c);
    const bool shE = lane != 31 && nb[0] == c + 1;
    const bool shW = lane != 0 && nb[1] == c - 1;
    const bool shWf = shW && fo[1] == __ldg(L.fof + (c > 0 ? c - 1 : 0));
    const unsigned tvo = (unsigned)c + (upper ? 0u : ncol);   // the vertical face ahead of the walk
    auto slot = [&](int j, int w) -> float* { return ring + ((size_t)j * NW + w) * bd + tid; };
    auto stage = [&](int i) {
        const int j = i % DEEP;
        const unsigned kc = kc0 + (unsigned)i * dkc, kcc = kcc0 + (unsigned)i * dkcc;
        if (BD) __pipeline_memcpy_async(rbd + (size_t)j * bd + tid, b + (kc + c), 8);
        else __pipeline_memcpy_async(slot(j, W_B), b + (kc + c), 4);
        __pipeline_memcpy_async(slot(j, W_TE), L.Th + (2 * kc + fo[0]), 4);
        __pipeline_memcpy_async(slot(j, W_TN), L.Th + (2 * kc + fo[2]), 4);
        __pipeline_memcpy_async(slot(j, W_TV), L.Tv + (kc + tvo), 4);
        __pipeline_memcpy_async(slot(j, W_TS), L.Th + (2 * kc + fo[3]), 4);
        if (!shWf) __pipeline_memcpy_async(slot(j, W_TW), L.Th + (2 * kc + fo[1]), 4);
        if (RAW) {
            __pipeline_memcpy_async(slot(j, W_XN), x + (kc + dkc + c), 4);
            __pipeline_memcpy_async(slot(j, W_XNB), x + (kc + nb[2]), 4);
            __pipeline_memcpy_async(slot(j, W_XS), x + (kc + nb[3]), 4);
            if (!shE) __pipeline_memcpy_async(slot(j, W_XE), x + (kc + nb[0]), 4);
            if (!shW) __pipeline_memcpy_async(slot(j, W_XW), x + (kc + nb[1]), 4);
        }
        if (PRO) {
            __pipeline_memcpy_async(slot(j, W_CN), xc + (kcc + dkcc + pc), 4);
            __pipeline_memcpy_async(slot(j, W_CNB), xc + (kcc + pn[2]), 4);
            __pipeline_memcpy_async(slot(j, W_CS), xc + (kcc + pn[3]), 4);
            if (!shE) __pipeline_memcpy_async(slot(j, W_CE), xc + (kcc + pn[0]), 4);
            if (!shW) __pipeline_memcpy_async(slot(j, W_CW), xc + (kcc + pn[1]), 4);
        }
    };
#pragma unroll
    for (int i = 0; i < DEEP; ++i) {
        if (i < NS) stage(i);
        __pipeline_commit();
    }
    float xprev = 0.f, x0 = 0.f, tprev = 0.f;
    if (RAW) x0 = __ldg(x + kc0 + c);
    if (PRO) x0 += __ldg(xc + kcc0 + pc);
    float q = 0.f, ip = 0.f, y = 0.f, anext = 0.f;
    float sw[NS], se[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int j = i % DEEP;
        __pipeline_wait_prior(DEEP - 1);
        __syncwarp();   // every lane's copies of this slot are complete and visible
        const float bk = BD ? (float)rbd[(size_t)j * bd + tid] : *slot(j, W_B);
        const float te = *slot(j, W_TE), tn = *slot(j, W_TN), tv = *slot(j, W_TV), ts = *slot(j, W_TS);
        const float tw = shWf ? ring[((size_t)j * NW + W_TE) * bd + tid - 1] : *slot(j, W_TW);
        float xn = 0.f, xh[4] = {0.f, 0.f, 0.f, 0.f};
        if (RAW) {
            xn = *slot(j, W_XN);
            xh[0] = *slot(j, W_XE);
            xh[1] = *slot(j, W_XW);
            xh[2] = *slot(j, W_XNB);
            xh[3] = *slot(j, W_XS);
        }
        if (PRO) {
            xn += *slot(j, W_CN);
            xh[0] += *slot(j, W_CE);
            xh[1] += *slot(j, W_CW);
            xh[2] += *slot(j, W_CNB);
            xh[3] += *slot(j, W_CS);
        }
        __syncwarp();   // reads of the slot are done before it is refilled
        if (i + DEEP < NS) stage(i + DEEP);
        __pipeline_commit();
        const float xEl = __shfl_down_sync(0xffffffffu, x0, 1);
        const float xWl = __shfl_up_sync(0xffffffffu, x0, 1);
        if (shE) xh[0] = xEl;
        if (shW) xh[1] = xWl;
        const float rdz = srdz[kfirst + dir * i];
        if (BCOPY) bcopy[kc0 + (unsigned)i * dkc + c] = bk;
        float r = bk;
        if (MODE != XM_ZERO) {
            float hx = te * (x0 - xh[0]);
            hx += tw * (x0 - xh[1]);
            hx += tn * (x0 - xh[2]);
            hx += ts * (x0 - xh[3]);
            r -= x0 + (rA * hx + rdz * (tv * (x0 - xn) + tprev * (x0 - xprev)));
        }
        anext = rdz * tv;
        const float m = (rdz * tprev) * ip;
        q = (1.f + rA * ((te + tw) + (tn + ts))) + m * q;
        const float p = q + anext;
        y = r + m * y;
        ip = 1.f / p;
        const float ei = anext * ip;
        sw[i] = x0 + omega * (y * ip) - ei * xn;
        se[i] = ei;
        xprev = x0;
        x0 = xn;
        tprev = tv;
    }
    __pipeline_wait_prior(0);
    // interface rows: through shared memory from the thread tid ^ (bd / 2) holding the other half
    __syncthreads();
    float* xch = reinterpret_cast<float*>(smem_raw);
    xch[tid] = q;
    xch[bd + tid] = y;
    xch[2 * bd + tid] = anext;
    __syncthreads();
    const int pt = tid ^ (bd >> 1);
    const float qo = xch[pt], yo = xch[bd + pt], ao = xch[2 * bd + pt];
    const float po = qo + ao;
    const float dlt = (y * po + anext * yo) / (q * po + anext * qo);
    if (!active) return;
    float out = xprev + omega * dlt;
    O* pout = xo + c;
    unsigned ko = kc0 + (unsigned)(NS - 1) * dkc;
    pout[ko] = (O)out;
#pragma unroll
    for (int i = NS - 2; i >= 0; --i) {
        out = sw[i] + se[i] * out;
        ko -= dkc;
        pout[ko] = (O)out;
    }
}

// ---------------------------------------------------------------------------------------
// Residual and restriction (Algorithm 1): bc[k][C] = sum_q w[q][C] (b - H x)[k][child_q],
// w = area_child / area_C; one thread per coarse column and chunk of kchunk levels (there is
// no vertical recurrence, so short chunks give many independent threads).
template <typename T, typename C, bool XZERO, typename X, typename B, typename O>
__global__ void __launch_bounds__(128) k_resid_restrict(Lvl<T, C> L, const X* __restrict__ x,
                                                         const B* __restrict__ b,
                                                         const T* __restrict__ w,
                                                         O* __restrict__ bc, int ncol_c, int kchunk) {
    const int Cc = blockIdx.x * blockDim.x + threadIdx.x;
    if (Cc >= ncol_c) return;
    const size_t ncol = L.ncol, nf = 2 * ncol;
    const int k0 = blockIdx.y * kchunk;
    const int k1 = min(L.nlev, k0 + kchunk);
    int ch[4], nb[4][4], fo[4][4];
    T rA[4], wq[4], xm[4], x0[4], tdn[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        ch[q] = child_col_dev(L.n, Cc, q);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            nb[q][s] = __ldg(L.nbr + s * ncol + ch[q]);
            fo[q][s] = __ldg(L.fof + s * ncol + ch[q]);
        }
        rA[q] = __ldg(L.rA + ch[q]);
        wq[q] = __ldg(w + (size_t)q * ncol_c + Cc);
        xm[q] = (XZERO || k0 == 0) ? T(0) : ldx<T>(x + (size_t)(k0 - 1) * ncol + ch[q]);
        x0[q] = XZERO ? T(0) : ldx<T>(x + (size_t)k0 * ncol + ch[q]);
        tdn[q] = ldc<T>(L.Tv + (size_t)k0 * ncol + ch[q]);
    }
    for (int k = k0; k < k1; ++k) {
        const size_t o = (size_t)k * ncol;
        const C* th = L.Th + (size_t)k * nf;
        const T rdz = __ldg(L.rdz + k);
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T tup = ldc<T>(L.Tv + o + ncol + ch[q]);
            T r = (T)__ldg(b + o + ch[q]);
            if (!XZERO) {
                const T xp = (k + 1 < L.nlev) ? ldx<T>(x + o + ncol + ch[q]) : T(0);
                T h = ldc<T>(th + fo[q][0]) * (x0[q] - ldx<T>(x + o + nb[q][0]));
                h += ldc<T>(th + fo[q][1]) * (x0[q] - ldx<T>(x + o + nb[q][1]));
                h += ldc<T>(th + fo[q][2]) * (x0[q] - ldx<T>(x + o + nb[q][2]));
                h += ldc<T>(th + fo[q][3]) * (x0[q] - ldx<T>(x + o + nb[q][3]));
                r -= x0[q] + (rA[q] * h + rdz * (tup * (x0[q] - xp) + tdn[q] * (x0[q] - xm[q])));
                xm[q] = x0[q];
                x0[q] = xp;
            }
            tdn[q] = tup;
            acc += wq[q] * r;
        }
        bc[(size_t)k * ncol_c + Cc] = (O)acc;
    }
}

// Residual and restriction, one thread per fine column (for n divisible by 16): a warp
// covers fine columns i0..i0+15 of rows 2J (lanes 0-15) and 2J+1 (lanes 16-31) of one
// panel, i.e. 8 coarse columns; the 2x2 sums of w_child r_child are two shuffles, and the
// E / W neighbour iterates and the W face come from the adjacent lanes.  Each thread walks
// kchunk levels with loads issued SHAL levels ahead in a register ring.
template <typename T, typename C, bool XZERO, typename X, typename B, typename O, int SHAL>
__global__ void __launch_bounds__(128) k_resid_restrict16(Lvl<T, C> L, const X* __restrict__ x,
                                                           const B* __restrict__ b,
                                                           const T* __restrict__ w,
                                                           O* __restrict__ bc, int ncol_c, int kchunk) {
    const int n = L.n, nc = n >> 1, tiles = n >> 4;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nwarps = 6 * nc * tiles;   // (panel, coarse row, tile)
    const int lane = threadIdx.x & 31;
    const bool valid = warp < nwarps;
    const int wq = valid ? warp : 0;
    const int p = wq / (nc * tiles), rem = wq - p * nc * tiles, J = rem / tiles, t = rem - J * tiles;
    const int rowf = 2 * J + (lane >> 4), i = t * 16 + (lane & 15);
    const int c = p * n * n + rowf * n + i;
    const int Cc = p * nc * nc + J * nc + (i >> 1);
    const int q = ((lane >> 4) << 1) | (i & 1);   // child index 2b + a
    const size_t ncol = L.ncol, nf = 2 * ncol;
    const int k0 = blockIdx.y * kchunk;
    const int k1 = min(L.nlev, k0 + kchunk);
    int nb[4], fo[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        nb[s] = __ldg(L.nbr + s * ncol + c);
        fo[s] = __ldg(L.fof + s * ncol + c);
    }
    const T rA = __ldg(L.rA + c);
    const T wc = __ldg(w + (size_t)q * ncol_c + Cc);
    // E / W neighbours that are the adjacent lanes of the 16-lane row group: their iterate
    // and (W) face coefficient come by shuffle instead of a load
    const int gl = lane & 15;
    const bool shE = gl != 15 && nb[0] == c + 1;
    const bool shW = gl != 0 && nb[1] == c - 1;
    const bool shWf = shW && fo[1] == __ldg(L.fof + (c > 0 ? c - 1 : 0));
    struct Lv {
        T xp, xn[4], b, th[4], tup, rdz;
    };
    auto load = [&](int k, Lv& d) {
        const size_t o = (size_t)k * ncol;
        if (!XZERO) {
            d.xp = (k + 1 < L.nlev) ? ldx<T>(x + o + ncol + c) : T(0);
            if (!shE) d.xn[0] = ldx<T>(x + o + nb[0]);
            if (!shW) d.xn[1] = ldx<T>(x + o + nb[1]);
            d.xn[2] = ldx<T>(x + o + nb[2]);
            d.xn[3] = ldx<T>(x + o + nb[3]);
        }
        const C* th = L.Th + (size_t)k * nf;
        d.th[0] = ldc<T>(th + fo[0]);
        if (!shWf) d.th[1] = ldc<T>(th + fo[1]);
        d.th[2] = ldc<T>(th + fo[2]);
        d.th[3] = ldc<T>(th + fo[3]);
        d.tup = ldc<T>(L.Tv + o + ncol + c);
        d.b = (T)__ldg(b + o + c);
        d.rdz = __ldg(L.rdz + k);
    };
    Lv ring[SHAL];
#pragma unroll
    for (int j = 0; j < SHAL; ++j)
        if (k0 + j < k1) load(k0 + j, ring[j]);
    T xm = (XZERO || k0 == 0) ? T(0) : ldx<T>(x + (size_t)(k0 - 1) * ncol + c);
    T x0 = XZERO ? T(0) : ldx<T>(x + (size_t)k0 * ncol + c);
    T tdn = ldc<T>(L.Tv + (size_t)k0 * ncol + c);
    for (int kb = k0; kb < k1; kb += SHAL) {
#pragma unroll
        for (int j = 0; j < SHAL; ++j) {
            const int k = kb + j;
            if (k < k1) {
                const Lv d = ring[j];
                if (k + SHAL < k1) load(k + SHAL, ring[j]);
                const T twl = __shfl_up_sync(0xffffffffu, d.th[0], 1);
                const T xEl = __shfl_down_sync(0xffffffffu, x0, 1);
                const T xWl = __shfl_up_sync(0xffffffffu, x0, 1);
                const T tw = shWf ? twl : d.th[1];
                T r = d.b;
                if (!XZERO) {
                    const T xE = shE ? xEl : d.xn[0];
                    const T xW = shW ? xWl : d.xn[1];
                    T h = d.th[0] * (x0 - xE);
                    h += tw * (x0 - xW);
                    h += d.th[2] * (x0 - d.xn[2]);
                    h += d.th[3] * (x0 - d.xn[3]);
                    r -= x0 + (rA * h + d.rdz * (d.tup * (x0 - d.xp) + tdn * (x0 - xm)));
                    xm = x0;
                    x0 = d.xp;
                }
                tdn = d.tup;
                // sum the 4 children in the order (a=0,b=0)+(a=1,b=0) + (a=0,b=1)+(a=1,b=1)
                T v = wc * r;
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 16);
                if (valid && (lane & 17) == 0) bc[(size_t)k * ncol_c + Cc] = (O)v;
            }
        }
    }
}

// The same residual and restriction for FP32 levels with the own column's streams (b, the
// iterate one level up, the E and N faces and the vertical face above) copied DEEP levels
// ahead into a per-thread shared-memory ring by asynchronous 4-byte copies, which hold no
// registers while in flight; the neighbour iterates, the W and S faces and 1/dz stay in a
// SHAL-deep register ring.  Same warp layout and arithmetic order as k_resid_restrict16.
template <int DEEP, int SHAL>
__global__ void __launch_bounds__(128) k_resid_restrict16a(Lvl<float, float> L, const float* __restrict__ x,
                                                            const float* __restrict__ b,
                                                            const float* __restrict__ w, float* __restrict__ bc,
                                                            int ncol_c, int kchunk) {
    static_assert(DEEP % SHAL == 0, "ring lengths");
    __shared__ float ring[5][DEEP][128];   // b, x one level up, E face, N face, vertical face above
    const int n = L.n, nc = n >> 1, tiles = n >> 4;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nwarps = 6 * nc * tiles;   // (panel, coarse row, tile)
    const int lane = threadIdx.x & 31, tid = threadIdx.x;
    const bool valid = warp < nwarps;
    const int wq = valid ? warp : 0;
    const int p = wq / (nc * tiles), rem = wq - p * nc * tiles, J = rem / tiles, t = rem - J * tiles;
    const int rowf = 2 * J + (lane >> 4), i = t * 16 + (lane & 15);
    const int c = p * n * n + rowf * n + i;
    const int Cc = p * nc * nc + J * nc + (i >> 1);
    const int q = ((lane >> 4) << 1) | (i & 1);   // child index 2b + a
    const size_t ncol = L.ncol, nf = 2 * ncol;
    const int nlev = L.nlev;
    const int k0 = blockIdx.y * kchunk;
    const int k1 = min(nlev, k0 + kchunk);
    int nb[4], fo[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        nb[s] = __ldg(L.nbr + s * ncol + c);
        fo[s] = __ldg(L.fof + s * ncol + c);
    }
    const float rA = __ldg(L.rA + c);
    const float wc = __ldg(w + (size_t)q * ncol_c + Cc);
    const int gl = lane & 15;
    const bool shE = gl != 15 && nb[0] == c + 1;
    const bool shW = gl != 0 && nb[1] == c - 1;
    const bool shWf = shW && fo[1] == __ldg(L.fof + (c > 0 ? c - 1 : 0));
    auto stage = [&](int k, int slot) {
        if (k < k1) {
            const size_t o = (size_t)k * ncol;
            const bool in = k + 1 < nlev;
            __pipeline_memcpy_async(&ring[0][slot][tid], b + o + c, 4);
            __pipeline_memcpy_async(&ring[1][slot][tid], x + (in ? o + ncol : o) + c, 4, in ? 0 : 4);
            __pipeline_memcpy_async(&ring[2][slot][tid], L.Th + (size_t)k * nf + fo[0], 4);
            __pipeline_memcpy_async(&ring[3][slot][tid], L.Th + (size_t)k * nf + fo[2], 4);
            __pipeline_memcpy_async(&ring[4][slot][tid], L.Tv + o + ncol + c, 4);   // row nlev is zero
        }
        __pipeline_commit();
    };
    struct Lv {
        float xn[4], tw, ts, rdz;
    };
    auto load = [&](int k, Lv& d) {
        const size_t o = (size_t)k * ncol;
        if (!shE) d.xn[0] = __ldg(x + o + nb[0]);
        if (!shW) d.xn[1] = __ldg(x + o + nb[1]);
        d.xn[2] = __ldg(x + o + nb[2]);
        d.xn[3] = __ldg(x + o + nb[3]);
        if (!shWf) d.tw = __ldg(L.Th + (size_t)k * nf + fo[1]);
        d.ts = __ldg(L.Th + (size_t)k * nf + fo[3]);
        d.rdz = __ldg(L.rdz + k);
    };
#pragma unroll
    for (int j = 0; j < DEEP; ++j) stage(k0 + j, j);
    Lv rr[SHAL];
#pragma unroll
    for (int j = 0; j < SHAL; ++j)
        if (k0 + j < k1) load(k0 + j, rr[j]);
    float xm = k0 == 0 ? 0.f : __ldg(x + (size_t)(k0 - 1) * ncol + c);
    float x0 = __ldg(x + (size_t)k0 * ncol + c);
    float tdn = __ldg(L.Tv + (size_t)k0 * ncol + c);
    for (int kb = k0; kb < k1; kb += DEEP) {
#pragma unroll
        for (int j = 0; j < DEEP; ++j) {
            const int k = kb + j;
            __pipeline_wait_prior(DEEP - 1);
            __syncwarp();   // every lane's copies of this slot are complete and visible
            const float bk = ring[0][j][tid], xp = ring[1][j][tid], te = ring[2][j][tid], tn = ring[3][j][tid],
                        tup = ring[4][j][tid];
            __syncwarp();   // reads of the slot are done before it is refilled
            stage(k + DEEP, j);
            if (k < k1) {   // uniform over the block
                const Lv d = rr[j % SHAL];
                if (k + SHAL < k1) load(k + SHAL, rr[j % SHAL]);
                const float twl = __shfl_up_sync(0xffffffffu, te, 1);
                const float xEl = __shfl_down_sync(0xffffffffu, x0, 1);
                const float xWl = __shfl_up_sync(0xffffffffu, x0, 1);
                const float tw = shWf ? twl : d.tw;
                const float xE = shE ? xEl : d.xn[0];
                const float xW = shW ? xWl : d.xn[1];
                float h = te * (x0 - xE);
                h += tw * (x0 - xW);
                h += tn * (x0 - d.xn[2]);
                h += d.ts * (x0 - d.xn[3]);
                float r = bk;
                r -= x0 + (rA * h + d.rdz * (tup * (x0 - xp) + tdn * (x0 - xm)));
                xm = x0;
                x0 = xp;
                tdn = tup;
                float v = wc * r;
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 16);
                if (valid && (lane & 17) == 0) bc[(size_t)k * ncol_c + Cc] = v;
            }
        }
    }
    __pipeline_wait_prior(0);
}

// x_out[k][c] = (ZB ? 0 : x[k][c]) + xc[k][parent(c)]  (Eq. prolongation, natural injection)
template <typename T, bool ZB, typename X, typename O>
__global__ void k_prolong(int n, int ncol, int ncol_c, int nlev, const X* __restrict__ x,
                          const T* __restrict__ xc, O* __restrict__ xo) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    const int pc = parent_col(c, n);
    for (int k = 0; k < nlev; ++k) {
        const size_t o = (size_t)k * ncol;
        T v = __ldg(xc + (size_t)k * ncol_c + pc);
        if (!ZB) v += ldx<T>(x + o + c);
        xo[o + c] = (O)v;
    }
}

// ---------------------------------------------------------------------------------------
// The 9-cell stencil (Sec. 3.5, Fig. 2): H also couples every cell to the cells two levels
// above and below, through the fluxes T2[k][c] (k <-> k+2; rows nlev-2 and nlev-1 are zero):
// b_up(k) = T2[k] / dz_k, b_dn(k) = T2[k-2] / dz_k.  These kernels run one thread per cell or
// per column without staging: the 9-cell stencil is the paper's comparison configuration,
// not the headline path.
template <typename T, typename X>
__device__ __forceinline__ T h9_cell(const Lvl<T, T>& L, const T* __restrict__ T2, const X* __restrict__ x, int k,
                                     int c) {
    const size_t ncol = L.ncol, o = (size_t)k * ncol;
    const T x0 = ldx<T>(x + o + c);
    const T* th = L.Th + (size_t)k * 2 * ncol;
    T h = T(0);
#pragma unroll
    for (int s = 0; s < 4; ++s) h += __ldg(th + __ldg(L.fof + s * ncol + c)) * (x0 - ldx<T>(x + o + __ldg(L.nbr + s * ncol + c)));
    T v = T(0);
    if (k + 1 < L.nlev) v += __ldg(L.Tv + o + ncol + c) * (x0 - ldx<T>(x + o + ncol + c));
    if (k > 0) v += __ldg(L.Tv + o + c) * (x0 - ldx<T>(x + o - ncol + c));
    if (k + 2 < L.nlev) v += __ldg(T2 + o + c) * (x0 - ldx<T>(x + o + 2 * ncol + c));
    if (k > 1) v += __ldg(T2 + o - 2 * ncol + c) * (x0 - ldx<T>(x + o - 2 * ncol + c));
    return x0 + (__ldg(L.rA + c) * h + __ldg(L.rdz + k) * v);
}

// y = H x (9-cell stencil), one thread per cell
template <typename T, typename X, typename Y>
__global__ void k_apply9(Lvl<T, T> L, const T* __restrict__ T2, const X* __restrict__ x, Y* __restrict__ y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (c >= L.ncol || k >= L.nlev) return;
    y[(size_t)k * L.ncol + c] = (Y)h9_cell<T, X>(L, T2, x, k, c);
}

// r = b - H x (9-cell stencil; x == NULL: r = b), one thread per cell
template <typename T, typename B>
__global__ void k_resid9(Lvl<T, T> L, const T* __restrict__ T2, const T* __restrict__ x, const B* __restrict__ b,
                         T* __restrict__ r) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (c >= L.ncol || k >= L.nlev) return;
    const size_t e = (size_t)k * L.ncol + c;
    r[e] = x ? (T)b[e] - h9_cell<T, T>(L, T2, x, k, c) : (T)b[e];
}

// x_out = x + omega Hz^-1 r per column (x == NULL: zero iterate), Hz the tridiagonal column
// matrix of the nearest couplings (the next-to-nearest fluxes dropped, Sec. 3.6), solved by
// the pivot-excess Thomas recurrence; sw, se hold its y / p and a_up / p per cell
template <typename T, typename O>
__global__ void k_thomas9(Lvl<T, T> L, const T* __restrict__ r, const T* __restrict__ x, T* __restrict__ sw,
                          T* __restrict__ se, O* __restrict__ xo, T omega) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.ncol) return;
    const size_t ncol = L.ncol;
    const T rA = __ldg(L.rA + c);
    T q = T(0), p = T(1), y = T(0);
    for (int k = 0; k < L.nlev; ++k) {
        const size_t o = (size_t)k * ncol, e = o + c;
        const T* thk = L.Th + (size_t)k * 2 * ncol;
        T sh = T(0);
#pragma unroll
        for (int s = 0; s < 4; ++s) sh += __ldg(thk + __ldg(L.fof + s * ncol + c));
        const T rdz = __ldg(L.rdz + k);
        const T adn = k > 0 ? rdz * __ldg(L.Tv + e) : T(0);
        const T aup = k + 1 < L.nlev ? rdz * __ldg(L.Tv + e + ncol) : T(0);
        const T m = k > 0 ? adn / p : T(0);
        q = (T(1) + rA * sh) + m * q;
        p = q + aup;
        y = r[e] + m * y;
        sw[e] = y / p;
        se[e] = aup / p;
    }
    T d = T(0);
    for (int k = L.nlev - 1; k >= 0; --k) {
        const size_t e = (size_t)k * ncol + c;
        d = sw[e] + se[e] * d;
        xo[e] = (O)((x ? x[e] : T(0)) + omega * d);
    }
}

// bc[k][C] = sum_q w[q][C] r[k][child_q] (restriction of a residual already formed)
template <typename T, typename O>
__global__ void k_restrict_sum(int n, int ncol, int nlev, const T* __restrict__ r, const T* __restrict__ w,
                               O* __restrict__ bc, int ncol_c) {
    const int C = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (C >= ncol_c || k >= nlev) return;
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc += __ldg(w + (size_t)q * ncol_c + C) * r[(size_t)k * ncol + child_col_dev(n, C, q)];
    bc[(size_t)k * ncol_c + C] = (O)acc;
}

template <typename A, typename B>
__global__ void k_convert(size_t n, const A* __restrict__ a, B* __restrict__ b) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = (B)a[i];
}

}  // namespace mg
