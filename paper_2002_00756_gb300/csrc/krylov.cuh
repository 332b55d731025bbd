// FP64 vector kernels of the outer GCR iteration (Sec. 4.1 solver framework: axpy and
// inner products of the abstract vector type) and of the mixed system (Sec. 3.3-3.4).
//
// Inner products use a fixed grid, a fixed in-block shuffle tree and a last-block final
// sum in block order, so every run of the same launch gives bitwise the same scalars.
// The last block is found with a ticket counter (no block ever waits on another).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mg {

constexpr int RED_THREADS = 256;
constexpr int MAXR = 16;   // maximum GCR restart length (MG_MAX_RESTART)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Sums v[0..ND) over the whole grid; returns true in the one block that holds the totals,
// which thread 0 finds in `result`.
template <int ND>
__device__ bool grid_reduce(double (&v)[ND], double* partials, unsigned int* ticket, double* result) {
    __shared__ double sm[ND][RED_THREADS / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < ND; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < ND; ++i) sm[i][wid] = v[i];
    }
    __syncthreads();
    if (threadIdx.x < ND) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sm[threadIdx.x][w];
        partials[(size_t)blockIdx.x * ND + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    if (threadIdx.x < ND) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(partials + (size_t)b * ND + threadIdx.x);
        result[threadIdx.x] = s;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    __syncthreads();
    return true;
}

// sc[0] = <a, b>
__global__ void __launch_bounds__(RED_THREADS) k_dot(size_t n, const double* __restrict__ a,
                                                     const double* __restrict__ b, double* partials,
                                                     unsigned int* ticket, double* sc) {
    double v[1] = {0.0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v[0] += a[i] * b[i];
    grid_reduce<1>(v, partials, ticket, sc);
}

// dots[j] = <w, W_j>, j < s  (classical Gram-Schmidt coefficients, one pass over w)
__global__ void __launch_bounds__(RED_THREADS) k_gcr_dots(size_t n, const double* __restrict__ w,
                                                          const double* __restrict__ Wb, size_t ld, int s,
                                                          double* partials, unsigned int* ticket,
                                                          double* dots) {
    double v[MAXR];
#pragma unroll
    for (int j = 0; j < MAXR; ++j) v[j] = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int j = 0; j < MAXR; ++j)
            if (j < s) v[j] += wi * __ldg(Wb + (size_t)j * ld + i);
    }
    grid_reduce<MAXR>(v, partials, ticket, dots);
}

// w -= sum_j beta_j W_j, z -= sum_j beta_j Z_j, beta_j = dots[j] / ww[j]; then
// ww[s] = <w, w> and alpha = <r, w> / <w, w>.
__global__ void __launch_bounds__(RED_THREADS) k_gcr_orth(size_t n, double* __restrict__ w,
                                                          double* __restrict__ z,
                                                          const double* __restrict__ Wb,
                                                          const double* __restrict__ Zb, size_t ld, int s,
                                                          const double* __restrict__ dots, double* ww,
                                                          const double* __restrict__ r, double* partials,
                                                          unsigned int* ticket, double* tmp2,
                                                          double* alpha) {
    double beta[MAXR];
#pragma unroll
    for (int j = 0; j < MAXR; ++j) beta[j] = (j < s) ? dots[j] / ww[j] : 0.0;
    double v[2] = {0.0, 0.0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double wi = w[i], zi = z[i];
#pragma unroll
        for (int j = 0; j < MAXR; ++j) {
            if (j < s) {
                wi -= beta[j] * __ldg(Wb + (size_t)j * ld + i);
                zi -= beta[j] * __ldg(Zb + (size_t)j * ld + i);
            }
        }
        if (s > 0) {
            w[i] = wi;
            z[i] = zi;
        }
        v[0] += wi * wi;
        v[1] += __ldg(r + i) * wi;
    }
    if (grid_reduce<2>(v, partials, ticket, tmp2) && threadIdx.x == 0) {
        ww[s] = tmp2[0];
        *alpha = tmp2[1] / tmp2[0];
    }
}

// x += alpha z, r -= alpha w, rr = <r, r>
__global__ void __launch_bounds__(RED_THREADS) k_gcr_update(size_t n, double* __restrict__ x,
                                                            double* __restrict__ r,
                                                            const double* __restrict__ z,
                                                            const double* __restrict__ w,
                                                            const double* __restrict__ alpha,
                                                            double* partials, unsigned int* ticket,
                                                            double* rr) {
    const double a = *alpha;
    double v[1] = {0.0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        x[i] += a * __ldg(z + i);
        const double ri = r[i] - a * __ldg(w + i);
        r[i] = ri;
        v[0] += ri * ri;
    }
    grid_reduce<1>(v, partials, ticket, rr);
}

// ---------------------------------------------------------------------------------------
// Mixed system (u, p) kernels; see mgsolve.h for the velocity layout.
struct MixedDev {
    int ncol, nlev, nfh;            // nfh = 2 ncol horizontal faces per level
    const int32_t* faceL;           // [nfh]
    const int32_t* faceR;           // [nfh]
    const int32_t* fof;             // [4][ncol]
    const double* sdiv;             // [4][ncol] +-c_s dt (edge length / area), + if the column owns the face
    const double* kd_h;             // [nlev][nfh]   kappa_f / d_f, kappa_f = c_s dt g_f
    const double* kd_v;             // [nlev+1][ncol]
    const double* w_up;             // [nlev+1][ncol] eps beta_up (interior couplings only)
    const double* w_dn;             // [nlev+1][ncol]
    const double* mlump;            // [nlev+1][ncol] row sums of M-bar
    const double* divv;             // [nlev] c_s dt / dz
};

// (D u)_i, vertical velocities optionally divided by the lumped mass
template <bool LUMP>
__device__ __forceinline__ double div_cell(const MixedDev& M, int k, int c, const double* __restrict__ uh,
                                           const double* __restrict__ uv) {
    const size_t ncol = M.ncol;
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 4; ++d)
        s += __ldg(M.sdiv + d * ncol + c) * __ldg(uh + (size_t)k * M.nfh + __ldg(M.fof + d * ncol + c));
    double v = 0.0;
    if (k + 1 < M.nlev) {
        const size_t o = (size_t)(k + 1) * ncol + c;
        v += LUMP ? __ldg(uv + o) / __ldg(M.mlump + o) : __ldg(uv + o);
    }
    if (k > 0) {
        const size_t o = (size_t)k * ncol + c;
        v -= LUMP ? __ldg(uv + o) / __ldg(M.mlump + o) : __ldg(uv + o);
    }
    return s + __ldg(M.divv + k) * v;
}

// velocity rows on horizontal faces: yh = uh + kd (p_R - p_L)   [MODE 0]
// Step 3 on horizontal faces:         yh = uh - kd (p_R - p_L)   [MODE 1]
template <int MODE>
__global__ void k_mx_faces_h(MixedDev M, const double* __restrict__ uh, const double* __restrict__ p,
                             double* __restrict__ yh) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (f >= M.nfh) return;
    const size_t o = (size_t)k * M.nfh + f, op = (size_t)k * M.ncol;
    const double g = __ldg(M.kd_h + o) * (__ldg(p + op + __ldg(M.faceR + f)) - __ldg(p + op + __ldg(M.faceL + f)));
    yh[o] = MODE == 0 ? __ldg(uh + o) + g : __ldg(uh + o) - g;
}

// velocity rows on vertical faces: yv = M-bar uv + kd (p_kf - p_kf-1)   [MODE 0]
// Step 3 on vertical faces:         yv = (uv - kd (p_kf - p_kf-1)) / m  [MODE 1]
template <int MODE>
__global__ void k_mx_faces_v(MixedDev M, const double* __restrict__ uv, const double* __restrict__ p,
                             double* __restrict__ yv) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int kf = blockIdx.y;
    if (c >= M.ncol) return;
    const size_t ncol = M.ncol, o = (size_t)kf * ncol + c;
    if (kf == 0 || kf == M.nlev) {
        yv[o] = __ldg(uv + o);
        return;
    }
    const double g = __ldg(M.kd_v + o) * (__ldg(p + (size_t)kf * ncol + c) - __ldg(p + (size_t)(kf - 1) * ncol + c));
    if (MODE == 0) {
        yv[o] = __ldg(uv + o) + __ldg(M.w_up + o) * __ldg(uv + o + ncol) + __ldg(M.w_dn + o) * __ldg(uv + o - ncol) + g;
    } else {
        yv[o] = (__ldg(uv + o) - g) / __ldg(M.mlump + o);
    }
}

// pressure rows: yp = p + D u                           [MODE 0]
// Step 1:        B  = rp - D M-ring^{-1} ru (p := rp)    [MODE 1]
template <int MODE>
__global__ void k_mx_cells(MixedDev M, const double* __restrict__ uh, const double* __restrict__ uv,
                           const double* __restrict__ p, double* __restrict__ yp) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (c >= M.ncol) return;
    const size_t o = (size_t)k * M.ncol + c;
    if (MODE == 0) yp[o] = __ldg(p + o) + div_cell<false>(M, k, c, uh, uv);
    else yp[o] = __ldg(p + o) - div_cell<true>(M, k, c, uh, uv);
}

}  // namespace mg
