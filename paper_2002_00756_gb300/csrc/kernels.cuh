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
#include <cuda_runtime.h>
#include <stdint.h>

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
// One block-Jacobi sweep (Eq. jacobi): x_out = x + omega Hz^{-1} (b - H x), per column:
// forward pass computes the residual and eliminates with pivots p_k = q_k + a_up_k,
// q_k = s_k + (a_dn_k / p_{k-1}) q_{k-1} (s_k = 1 + horizontal coefficients, so no
// subtraction), stashing y_k / p_k and a_up_k / p_k in shared memory; the backward
// pass substitutes and writes x_out.  Optionally copies b into `bcopy` (entry of the
// FP32 V-cycle, where b arrives in FP64).
//
// Latency hiding: loads are issued ahead into register rings, indexed statically because
// the loop over k is unrolled by the ring length: the streams met first in DRAM (own
// column: x above, b, the E and N face coefficients, the face above) run DEEP levels
// ahead; the loads that mostly hit in cache (W and S faces, the four neighbour iterates,
// prolongation terms) run SHAL levels ahead.  The elimination recurrence then never waits
// on memory.
template <typename T>
struct SweepDeep {
    T xp, b, te, tn, tup;
};
template <typename T>
struct SweepShal {
    T xn[4], tw, ts, cp, cn[4];
};

template <typename T, typename C, int MODE, typename X, typename B, typename O, bool BCOPY, int DEEP, int SHAL>
__global__ void k_sweep(Lvl<T, C> L, const X* __restrict__ x, const T* __restrict__ xc,
                        int ncol_c, const B* __restrict__ b, T* __restrict__ bcopy,
                        O* __restrict__ xo, T omega) {
    static_assert(DEEP % SHAL == 0, "ring lengths");
    constexpr bool PRO = (MODE == XM_PROLONG || MODE == XM_PROLONG0);
    constexpr bool RAW = (MODE == XM_PLAIN || MODE == XM_PROLONG);   // reads the fine iterate
    extern __shared__ unsigned char smem_raw[];
    T* sc = reinterpret_cast<T*>(smem_raw);
    T* se = sc + (size_t)L.nlev * blockDim.x;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.ncol) return;
    const int tid = threadIdx.x, bd = blockDim.x, nlev = L.nlev;
    const size_t ncol = L.ncol, nf = 2 * ncol;
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

    auto load_deep = [&](int k, SweepDeep<T>& d) {
        const size_t o = (size_t)k * ncol;
        const C* th = L.Th + (size_t)k * nf;
        if (RAW) d.xp = (k + 1 < nlev) ? ldx<T>(x + o + ncol + c) : T(0);
        d.b = (T)__ldg(b + o + c);
        d.te = ldc<T>(th + fo[0]);
        d.tn = ldc<T>(th + fo[2]);
        d.tup = ldc<T>(L.Tv + o + ncol + c);
    };
    auto load_shal = [&](int k, SweepShal<T>& d) {
        const size_t o = (size_t)k * ncol, oc = (size_t)k * ncol_c;
        const C* th = L.Th + (size_t)k * nf;
        if (RAW) {
#pragma unroll
            for (int s = 0; s < 4; ++s) d.xn[s] = ldx<T>(x + o + nb[s]);
        }
        if (PRO) {
            d.cp = (k + 1 < nlev) ? __ldg(xc + oc + ncol_c + pc) : T(0);
#pragma unroll
            for (int s = 0; s < 4; ++s) d.cn[s] = __ldg(xc + oc + pn[s]);
        }
        d.tw = ldc<T>(th + fo[1]);
        d.ts = ldc<T>(th + fo[3]);
    };

    SweepDeep<T> dr[DEEP];
    SweepShal<T> sr[SHAL];
#pragma unroll
    for (int j = 0; j < DEEP; ++j)
        if (j < nlev) load_deep(j, dr[j]);
#pragma unroll
    for (int j = 0; j < SHAL; ++j)
        if (j < nlev) load_shal(j, sr[j]);
    T xm = T(0), x0 = T(0), tdn = T(0);
    if (RAW) x0 = ldx<T>(x + c);
    if (PRO) x0 += __ldg(xc + pc);
    T q = T(0), ip = T(0), y = T(0);
    for (int k0 = 0; k0 < nlev; k0 += DEEP) {
#pragma unroll
        for (int j = 0; j < DEEP; ++j) {
            const int k = k0 + j;
            if (k < nlev) {
                const SweepDeep<T> d = dr[j];
                const SweepShal<T> e = sr[j % SHAL];
                if (k + DEEP < nlev) load_deep(k + DEEP, dr[j]);
                if (k + SHAL < nlev) load_shal(k + SHAL, sr[j % SHAL]);
                T xp = T(0), xe[4] = {T(0), T(0), T(0), T(0)};
                if (RAW) {
                    xp = d.xp;
#pragma unroll
                    for (int s = 0; s < 4; ++s) xe[s] = e.xn[s];
                }
                if (PRO) {
                    xp += e.cp;
#pragma unroll
                    for (int s = 0; s < 4; ++s) xe[s] += e.cn[s];
                }
                const T rdz = __ldg(L.rdz + k);
                if (BCOPY) bcopy[(size_t)k * ncol + c] = d.b;
                T r = d.b;
                if (MODE != XM_ZERO) {
                    T hx = d.te * (x0 - xe[0]);
                    hx += e.tw * (x0 - xe[1]);
                    hx += d.tn * (x0 - xe[2]);
                    hx += e.ts * (x0 - xe[3]);
                    r -= x0 + (rA * hx + rdz * (d.tup * (x0 - xp) + tdn * (x0 - xm)));
                }
                const T aup = rdz * d.tup, adn = rdz * tdn;
                const T m = adn * ip;
                q = (T(1) + rA * ((d.te + e.tw) + (d.tn + e.ts))) + m * q;
                const T p = q + aup;
                y = r + m * y;
                ip = T(1) / p;
                sc[(size_t)k * bd + tid] = y * ip;
                se[(size_t)k * bd + tid] = aup * ip;
                xm = x0;
                x0 = xp;
                tdn = d.tup;
            }
        }
    }
    T dlt = T(0);
#pragma unroll 4
    for (int k = nlev - 1; k >= 0; --k) {
        dlt = sc[(size_t)k * bd + tid] + se[(size_t)k * bd + tid] * dlt;
        const size_t o = (size_t)k * ncol, oc = (size_t)k * ncol_c;
        xo[o + c] = (O)(xval<MODE, T>(x, xc, o, oc, c, pc) + omega * dlt);
    }
}

// ---------------------------------------------------------------------------------------
// Residual and restriction (Algorithm 1): bc[k][C] = sum_q w[q][C] (b - H x)[k][child_q],
// w = area_child / area_C; one thread per coarse column.
template <typename T, typename C, bool XZERO, typename X, typename B, typename O>
__global__ void __launch_bounds__(128) k_resid_restrict(Lvl<T, C> L, const X* __restrict__ x,
                                                         const B* __restrict__ b,
                                                         const T* __restrict__ w,
                                                         O* __restrict__ bc, int ncol_c) {
    const int Cc = blockIdx.x * blockDim.x + threadIdx.x;
    if (Cc >= ncol_c) return;
    const size_t ncol = L.ncol, nf = 2 * ncol;
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
        xm[q] = T(0);
        x0[q] = XZERO ? T(0) : ldx<T>(x + ch[q]);
        tdn[q] = T(0);
    }
    for (int k = 0; k < L.nlev; ++k) {
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

template <typename A, typename B>
__global__ void k_convert(size_t n, const A* __restrict__ a, B* __restrict__ b) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = (B)a[i];
}

}  // namespace mg
