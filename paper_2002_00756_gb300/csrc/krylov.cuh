// FP64 vector kernels of the outer GCR iteration (Sec. 4.1 solver framework: axpy and
// inner products of the abstract vector type) and of the mixed system (Sec. 3.3-3.4).
//
// Inner products use a fixed grid, a fixed in-block shuffle tree and a last-block final
// sum in block order, so every run of the same launch gives bitwise the same scalars.
// The last block is found with a ticket counter (no block ever waits on another).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

// fused GCR apply in diagonal form (1) or difference form (0)
#ifndef MG_APPLY_DIAG
#define MG_APPLY_DIAG 1
#endif

namespace mg {

constexpr int RED_THREADS = 256;
constexpr int MAXR = 16;   // maximum GCR restart length (MG_MAX_RESTART)

// device scalar block of the GCR iteration
struct GcrScal {
    double beta[MAXR * MAXR];   // beta[j * MAXR + i]: w_j orthogonalised against w_i, i < j
    double alpha[MAXR];         // step length of direction j
    double ww[MAXR];            // <w_i, w_i> of the orthogonalised directions
    double rr, bb;              // <r, r>, <b, b>
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Sums v[0..ND) over the whole grid (any 1-D or 2-D grid of RED_THREADS-thread blocks).
// Each block writes its ND partial sums; the last block to finish (ticket counter, no
// waiting) adds all partials with every thread taking a fixed stride of blocks, then a
// fixed tree; thread 0 of that block gets the totals in `tot` and the function returns
// true there.  The order of every addition is fixed, so results are bitwise repeatable.
template <int ND>
__device__ bool grid_reduce(double (&v)[ND], double* partials, unsigned int* ticket, double (&tot)[ND]) {
    __shared__ double sm[ND][RED_THREADS / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned nblk = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
    for (int i = 0; i < ND; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < ND; ++i) sm[i][wid] = v[i];
    }
    __syncthreads();
    if (threadIdx.x < ND) {
        double s = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) s += sm[threadIdx.x][w];
        partials[(size_t)bid * ND + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == nblk - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double a[ND];
#pragma unroll
    for (int i = 0; i < ND; ++i) a[i] = 0.0;
    for (unsigned b = threadIdx.x; b < nblk; b += RED_THREADS) {
#pragma unroll
        for (int i = 0; i < ND; ++i) a[i] += __ldcg(partials + (size_t)b * ND + i);
    }
#pragma unroll
    for (int i = 0; i < ND; ++i) a[i] = warp_sum(a[i]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < ND; ++i) sm[i][wid] = a[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < ND; ++i) {
            double s = 0.0;
            for (int w = 0; w < RED_THREADS / 32; ++w) s += sm[i][w];
            tot[i] = s;
        }
        *ticket = 0u;
    }
    return threadIdx.x == 0;
}

// out = V x (multiply) or V^-1 x, V = area[col] * dz[k] the finest level's cell volumes
__global__ void k_scale_volume(int ncol, int nlev, const double* __restrict__ area, const double* __restrict__ dz,
                               const double* x, double* out, bool multiply) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (c >= ncol || k >= nlev) return;
    const size_t e = (size_t)k * ncol + c;
    const double v = __ldg(area + c) * __ldg(dz + k);
    out[e] = multiply ? x[e] * v : x[e] / v;
}

// ---- caller-supplied couplings a[s][k][c] (s = E, W, N, S, up, down) of the finest level ----
// Their face form: Th[k][f] = a_(owner, side)(k) area(owner) (horizontal), Tv[kf][c] =
// a_up(kf-1, c) dz[kf-1] (vertical).  Valid only for a flux-symmetric operator, V_i a_if = V_j a_jf:
// the other cell's product must agree to 1e-10 relative, every coupling must be finite and
// >= 0, and none may cross the surface or the lid.  A failed check sets *bad; with write the
// kernels store the face form in every precision the handle holds (NULL arrays are skipped).
struct CoefTargets {
    double* Th64;
    float* Th32;
    __nv_bfloat16* Th16;
    double* Tv64;
    float* Tv32;
    __nv_bfloat16* Tv16;
};

__device__ __forceinline__ bool coef_close(double u, double v) {
    return fabs(u - v) <= 1e-10 * fmax(fabs(u), fabs(v));
}

__global__ void k_coef_faces(int ncol, int nlev, const int32_t* __restrict__ faceL, const int32_t* __restrict__ faceR,
                             const int32_t* __restrict__ faceSide, const int32_t* __restrict__ nbrSide,
                             const double* __restrict__ area, const double* __restrict__ a, bool write, CoefTargets t,
                             unsigned int* bad) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y, nf = 2 * ncol;
    if (f >= nf || k >= nlev) return;
    const size_t N = (size_t)nlev * ncol, o = (size_t)k * ncol;
    const int L = faceL[f], R = faceR[f], s = faceSide[f], sr = nbrSide[s * ncol + L];
    const double tl = a[s * N + o + L] * area[L], tr = a[sr * N + o + R] * area[R];
    if (!(tl >= 0.0) || !(tr >= 0.0) || !isfinite(tl) || !isfinite(tr) || !coef_close(tl, tr)) atomicOr(bad, 1u);
    if (!write) return;
    const size_t e = (size_t)k * nf + f;
    if (t.Th64) t.Th64[e] = tl;
    if (t.Th32) t.Th32[e] = (float)tl;
    if (t.Th16) t.Th16[e] = __float2bfloat16_rn((float)tl);
}

__global__ void k_coef_vertical(int ncol, int nlev, const double* __restrict__ dz, const double* __restrict__ a,
                                bool write, CoefTargets t, unsigned int* bad) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, kf = blockIdx.y;
    if (c >= ncol || kf > nlev) return;
    const size_t N = (size_t)nlev * ncol;
    double tv = 0.0;
    if (kf == 0) {
        if (a[5 * N + c] != 0.0) atomicOr(bad, 1u);                             // a_dn of the bottom cell
    } else if (kf == nlev) {
        if (a[4 * N + (size_t)(nlev - 1) * ncol + c] != 0.0) atomicOr(bad, 1u);  // a_up of the top cell
    } else {
        const double up = a[4 * N + (size_t)(kf - 1) * ncol + c], dn = a[5 * N + (size_t)kf * ncol + c];
        tv = up * dz[kf - 1];
        const double ta = dn * dz[kf];
        if (!(up >= 0.0) || !(dn >= 0.0) || !isfinite(tv) || !isfinite(ta) || !coef_close(tv, ta)) atomicOr(bad, 1u);
    }
    if (!write) return;
    const size_t e = (size_t)kf * ncol + c;
    if (t.Tv64) t.Tv64[e] = tv;
    if (t.Tv32) t.Tv32[e] = (float)tv;
    if (t.Tv16) t.Tv16[e] = __float2bfloat16_rn((float)tv);
}

// a6[s][e] = a[s][e] (s < 6) and a6[6][e] = 1 + their sum: the FP64 operator of the GCR apply
__global__ void k_coef_cells(size_t N, const double* __restrict__ a, double* __restrict__ a6) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x) {
        double d = 1.0;
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            const double v = a[s * N + e];
            a6[s * N + e] = v;
            d += v;
        }
        a6[6 * N + e] = d;
    }
}

// grad[s][e] = -lam_e (x_e - x_(neighbour s of e)), s = E, W, N, S, up, down (0 without a
// neighbour): the gradient of L(x) with respect to the six couplings of the finest level
__global__ void k_coef_grad(Lvl<double, double> L, const double* __restrict__ lam, const double* __restrict__ x,
                            double* __restrict__ grad) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (c >= L.ncol || k >= L.nlev) return;
    const size_t ncol = L.ncol, N = (size_t)L.nlev * ncol, e = (size_t)k * ncol + c;
    const double l = lam[e], x0 = x[e];
#pragma unroll
    for (int s = 0; s < 4; ++s) grad[s * N + e] = -l * (x0 - x[(size_t)k * ncol + __ldg(L.nbr + s * ncol + c)]);
    grad[4 * N + e] = k + 1 < L.nlev ? -l * (x0 - x[e + ncol]) : 0.0;
    grad[5 * N + e] = k > 0 ? -l * (x0 - x[e - ncol]) : 0.0;
}

// out = <a, b>
__global__ void __launch_bounds__(RED_THREADS) k_dot(size_t n, const double* __restrict__ a,
                                                     const double* __restrict__ b, double* partials,
                                                     unsigned int* ticket, double* out) {
    double v[1] = {0.0}, t[1];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v[0] += a[i] * b[i];
    if (grid_reduce<1>(v, partials, ticket, t)) *out = t[0];
}

// ---- BiCGStab for the pressure system (van der Vorst 1992, right-preconditioned) ----
// Device scalars of one solve: every vector kernel reads them, the last block of each
// reduction writes the ones it completes, and the host reads the block once per iteration.
struct BicgScal {
    double bb;              // <b, b>
    double rho, rho_old;    // <r^, r> of this step and of the one before
    double alpha, omega;
    double ss, rr;          // <s, s>, <r, r>
    double tol2bb;          // tol^2 <b, b>
    int half;               // ||s|| <= tol ||b||: the step ends after its first half
};

// y = H z on the finest level from the premultiplied couplings a6 (diagonal form, FP64)
__global__ void k_apply_a6(Lvl<double, double> L, const double* __restrict__ a6, const double* __restrict__ z,
                           double* __restrict__ w) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (c >= L.ncol || k >= L.nlev) return;
    const size_t ncol = L.ncol, N = (size_t)L.nlev * ncol, o = (size_t)k * ncol, e = o + c;
    double we = __ldg(a6 + 6 * N + e) * __ldg(z + e);
#pragma unroll
    for (int s = 0; s < 4; ++s) we = fma(-__ldg(a6 + s * N + e), __ldg(z + o + __ldg(L.nbr + s * ncol + c)), we);
    if (k + 1 < L.nlev) we = fma(-__ldg(a6 + 4 * N + e), __ldg(z + e + ncol), we);
    if (k > 0) we = fma(-__ldg(a6 + 5 * N + e), __ldg(z + e - ncol), we);
    w[e] = we;
}

#define MG_GRID_STRIDE(i, n) \
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

// r = r^ = b, x = 0; rho = <b, b>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_start(size_t n, const double* __restrict__ b, double* r,
                                                            double* rh, double* x, double tol, double* partials,
                                                            unsigned int* ticket, BicgScal* S) {
    double v[1] = {0.0}, t[1];
    MG_GRID_STRIDE(i, n) {
        const double bi = b[i];
        r[i] = bi;
        rh[i] = bi;
        x[i] = 0.0;
        v[0] += bi * bi;
    }
    if (grid_reduce<1>(v, partials, ticket, t)) {
        S->bb = t[0];
        S->rho = t[0];
        S->rho_old = 1.0;
        S->alpha = 1.0;
        S->omega = 1.0;
        S->tol2bb = tol * tol * t[0];
        S->half = 0;
    }
}

// p = r (first step) or p = r + (rho / rho_old)(alpha / omega)(p - omega v)
__global__ void k_bicg_dir(size_t n, const double* __restrict__ r, const double* __restrict__ v, double* p, bool first,
                           const BicgScal* S) {
    const double om = S->omega, beta = (S->rho / S->rho_old) * (S->alpha / om);
    MG_GRID_STRIDE(i, n) p[i] = first ? r[i] : r[i] + beta * (p[i] - om * v[i]);
}

// alpha = rho / <r^, v>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_alpha(size_t n, const double* __restrict__ rh,
                                                            const double* __restrict__ v, double* partials,
                                                            unsigned int* ticket, BicgScal* S) {
    double a[1] = {0.0}, t[1];
    MG_GRID_STRIDE(i, n) a[0] += rh[i] * v[i];
    if (grid_reduce<1>(a, partials, ticket, t)) S->alpha = S->rho / t[0];
}

// s = r - alpha v, <s, s>, and whether the step ends here
__global__ void __launch_bounds__(RED_THREADS) k_bicg_s(size_t n, const double* __restrict__ r,
                                                        const double* __restrict__ v, double* sv, double* partials,
                                                        unsigned int* ticket, BicgScal* S) {
    const double al = S->alpha;
    double a[1] = {0.0}, t[1];
    MG_GRID_STRIDE(i, n) {
        const double si = r[i] - al * v[i];
        sv[i] = si;
        a[0] += si * si;
    }
    if (grid_reduce<1>(a, partials, ticket, t)) {
        S->ss = t[0];
        S->half = t[0] <= S->tol2bb;
    }
}

// omega = <t, s> / <t, t>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_omega(size_t n, const double* __restrict__ tv,
                                                            const double* __restrict__ sv, double* partials,
                                                            unsigned int* ticket, BicgScal* S) {
    double a[2] = {0.0, 0.0}, t[2];
    MG_GRID_STRIDE(i, n) {
        a[0] += tv[i] * sv[i];
        a[1] += tv[i] * tv[i];
    }
    if (grid_reduce<2>(a, partials, ticket, t)) S->omega = t[0] / t[1];
}

// x += alpha p^ + omega s^, r = s - omega t (after a half step: x += alpha p^, r = s);
// then rho_old = rho, rho = <r^, r>, rr = <r, r>
__global__ void __launch_bounds__(RED_THREADS) k_bicg_xr(size_t n, double* x, double* r, const double* __restrict__ ph,
                                                         const double* __restrict__ sh, const double* __restrict__ sv,
                                                         const double* __restrict__ tv, const double* __restrict__ rh,
                                                         double* partials, unsigned int* ticket, BicgScal* S) {
    const double al = S->alpha, om = S->omega;
    const bool half = S->half != 0;
    double a[2] = {0.0, 0.0}, t[2];
    MG_GRID_STRIDE(i, n) {
        double ri;
        if (half) {
            x[i] += al * ph[i];
            ri = sv[i];
        } else {
            x[i] += al * ph[i] + om * sh[i];
            ri = sv[i] - om * tv[i];
        }
        r[i] = ri;
        a[0] += rh[i] * ri;
        a[1] += ri * ri;
    }
    if (grid_reduce<2>(a, partials, ticket, t)) {
        S->rho_old = S->rho;
        S->rho = t[0];
        S->rr = t[1];
    }
}

// ---- one graph launch for an ensemble of pressure solves ----
// Every member's GCR iterations run inside a conditional WHILE node of one CUDA graph; within
// it, an IF node per restart slot j holds the V-cycle, the fused apply and the orthogonalisation
// of slot j, and a second IF node the solution update that closes a restart cycle.  The
// decisions the host takes after each iteration of a single solve (converged, breakdown,
// iteration limit, end of a restart cycle) are taken here by one thread, in the same order
// and FP64 arithmetic, by setting the conditions of those nodes.
struct EnsState {
    double bb;     // <b, b>
    double rel;    // ||r|| / ||b|| after the last iteration
    int it;        // iterations done
    int status;    // MG_OK, MG_ERR_NOT_CONVERGED or MG_ERR_BREAKDOWN
};

struct EnsHandles {
    cudaGraphConditionalHandle w;          // WHILE: another iteration
    cudaGraphConditionalHandle c[MAXR];    // IF: iteration of slot j
    cudaGraphConditionalHandle x[MAXR];    // IF: solution update after slot j
};

// the device's global nanosecond clock
__global__ void k_stamp(unsigned long long* out) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    *out = t;
}

__device__ void ens_set_slots(const EnsHandles& hs, int R, int next, bool go) {
    for (int k = 0; k < R; ++k) {
        cudaGraphSetConditional(hs.c[k], (go && k == next) ? 1u : 0u);
        cudaGraphSetConditional(hs.x[k], 0u);
    }
}

// after <b, b>: start iterating unless b = 0, <b, b> is not finite or no iteration is allowed
__global__ void k_ens_init(const GcrScal* S, EnsState* st, int R, int max_iter, EnsHandles hs) {
    const double bb = S->bb;
    const bool bad = !isfinite(bb);
    const bool go = !bad && bb > 0.0 && max_iter > 0;
    st->bb = bb;
    st->it = 0;
    st->rel = (!bad && bb > 0.0) ? 1.0 : 0.0;
    st->status = bad ? MG_ERR_BREAKDOWN : (go ? MG_ERR_NOT_CONVERGED : MG_OK);
    ens_set_slots(hs, R, 0, go);
    cudaGraphSetConditional(hs.w, go ? 1u : 0u);
}

// after the iteration of slot j: the convergence test and the solution update of a single solve
__global__ void k_ens_decide(const GcrScal* S, EnsState* st, int j, int R, int max_iter, double tol, EnsHandles hs) {
    const int it = st->it + 1;
    st->it = it;
    const double rr = S->rr;
    if (!isfinite(rr)) {   // breakdown: stop without the update (x keeps the last cycle's value)
        st->status = MG_ERR_BREAKDOWN;
        ens_set_slots(hs, R, 0, false);
        cudaGraphSetConditional(hs.w, 0u);
        return;
    }
    const double rel = sqrt(rr / st->bb);
    st->rel = rel;
    const bool done = rel <= tol;
    if (done) st->status = MG_OK;
    const bool go = !done && it < max_iter;
    ens_set_slots(hs, R, j + 1 < R ? j + 1 : 0, go);
    cudaGraphSetConditional(hs.x[j], (j == R - 1 || done || it == max_iter) ? 1u : 0u);
    cudaGraphSetConditional(hs.w, go ? 1u : 0u);
}

// GCR step coefficients for direction J (classical Gram-Schmidt, one pass):
//   beta_i = <w, w_i> / <w_i, w_i>,  <w', w'> = <w, w> - sum_i beta_i <w, w_i>,
//   alpha = <r, w'> / <w', w'> with <r, w'> = <r, w> (the GCR residual is orthogonal to
//   all earlier directions w_i), from sums = [<w, w_i> (J), <w, w>, <r, w>].
// Every kernel below is instantiated for the exact number J of stored directions, so no
// FP64 instruction is spent on absent directions (FP64 issue rate bounds these kernels).
// <w', w'> is kept for the later directions' beta: the orthogonalisation pass does not
// recompute it (the FP64 pipe bounds that pass on GB300).
template <int J>
__device__ void gcr_coeffs(const double (&t)[J + 2], GcrScal* S) {
    double ww = t[J];
#pragma unroll
    for (int i = 0; i < J; ++i) {
        const double beta = t[i] / S->ww[i];
        S->beta[J * MAXR + i] = beta;
        ww -= beta * t[i];
    }
    S->ww[J] = ww;
    S->alpha[J] = t[J + 1] / ww;
}


template <int J>
__device__ __forceinline__ void gcr_accumulate(double (&v)[J + 2], double we, double re,
                                               const double* __restrict__ Wb, size_t ld, size_t e) {
#pragma unroll
    for (int i = 0; i < J; ++i) v[i] += we * __ldg(Wb + (size_t)i * ld + e);
    v[J] += we * we;
    v[J + 1] += re * we;
}

// GCR sums for a new direction w (mixed system path, where w comes from other kernels).
template <int J>
__global__ void __launch_bounds__(RED_THREADS) k_gcr_sums(size_t n, const double* __restrict__ w,
                                                          const double* __restrict__ Wb, size_t ld,
                                                          const double* __restrict__ r, double* partials,
                                                          unsigned int* ticket, GcrScal* S) {
    double v[J + 2], t[J + 2];
#pragma unroll
    for (int i = 0; i < J + 2; ++i) v[i] = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        gcr_accumulate<J>(v, __ldg(w + e), __ldg(r + e), Wb, ld, e);
    if (grid_reduce<J + 2>(v, partials, ticket, t)) gcr_coeffs<J>(t, S);
}

// w_J <- w_J - sum_i beta_i w_i (stored in place), r <- r - alpha_J w_J, then <r, r> -> rr
// (FP64: the residual spans the right-hand side's whole range, whose squares FP32 would
// flush to zero below about 1e-19).
template <int J>
__global__ void __launch_bounds__(RED_THREADS) k_gcr_orth_update(size_t n, double* __restrict__ Wb, size_t ld,
                                                                 double* __restrict__ r, double* partials,
                                                                 unsigned int* ticket, GcrScal* S) {
    double beta[J > 0 ? J : 1];
#pragma unroll
    for (int i = 0; i < J; ++i) beta[i] = S->beta[J * MAXR + i];
    const double a = S->alpha[J];
    double* w = Wb + (size_t)J * ld;
    double v[1] = {0.0}, t[1];
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double we = w[e];
#pragma unroll
        for (int i = 0; i < J; ++i) we -= beta[i] * __ldg(Wb + (size_t)i * ld + e);
        if (J > 0) w[e] = we;
        const double re = r[e] - a * we;
        r[e] = re;
        v[0] += re * re;
    }
    if (grid_reduce<1>(v, partials, ticket, t)) S->rr = t[0];
}

// x += sum_{i <= JL} gamma_i z_i with the raw (not orthogonalised) directions z_i:
// x = sum_i alpha_i zhat_i, zhat_i = z_i - sum_{m<i} beta_im zhat_m, unrolled from the top.
template <int JL>
__global__ void k_gcr_xupdate(size_t n, double* __restrict__ x, const double* __restrict__ Zb, size_t ld,
                              const GcrScal* __restrict__ S) {
    __shared__ double g[JL + 1];
    if (threadIdx.x == 0) {
        double a[JL + 1];
        for (int i = 0; i <= JL; ++i) a[i] = S->alpha[i];
        for (int i = JL; i >= 0; --i) {
            g[i] = a[i];
            for (int m = 0; m < i; ++m) a[m] -= a[i] * S->beta[i * MAXR + m];
        }
    }
    __syncthreads();
    double gr[JL + 1];
#pragma unroll
    for (int i = 0; i <= JL; ++i) gr[i] = g[i];
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double xe = x[e];
#pragma unroll
        for (int i = 0; i <= JL; ++i) xe += gr[i] * __ldg(Zb + (size_t)i * ld + e);
        x[e] = xe;
    }
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
    const double* rmlump;           // [nlev+1][ncol] 1 / row sums of M-bar
    const double* divv;             // [nlev] c_s dt / dz
    // horizontal faces: M_h u_f = ms u_f + sum_t wf[t][f] u_cf[t][f] (t < ncf), the same on
    // every level; lumped to 1 / rmlump_h
    int ncf;
    const int32_t* cf;              // [ncf][nfh]
    const double* wf;               // [ncf][nfh]
    double ms;                      // horizontal self weight
    double mv;                      // vertical self weight (interior faces)
    const double* rmlump_h;         // [nfh] 1 / lumped mass
    // adjoint: wfT[t][f] = weight of the entry of row cf[t][f] of M_h that points to f (the
    // rows of M_h^T), and the face weights W_f = A_f d_f / g_f on [u_h, u_v] (area dz / g of
    // the cell on the surface and lid faces), under which A^T = S J A-hat J S^-1 with S = diag(W, V)
    const double* wfT;              // [ncf][nfh]
    const double* Wf;               // [nlev][nfh] then [nlev+1][ncol]
    // coefficient gradient: d(kappa_f / d_f) / d g_i = c_s dt / (2 d_f) for both cells of f
    const double* cdh;              // [nfh]      c_s dt / (2 centre distance)
    const double* cdv;              // [nlev+1]   c_s dt / (2 dzc), 0 on surface and lid
    double eps;                     // strength of B_w
};

// (D u)_i, velocities optionally divided by the lumped mass
template <bool LUMP>
__device__ __forceinline__ double div_cell(const MixedDev& M, int k, int c, const double* __restrict__ uh,
                                           const double* __restrict__ uv) {
    const size_t ncol = M.ncol;
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int f = __ldg(M.fof + d * ncol + c);
        const double u = __ldg(uh + (size_t)k * M.nfh + f);
        s += __ldg(M.sdiv + d * ncol + c) * (LUMP ? u * __ldg(M.rmlump_h + f) : u);
    }
    double v = 0.0;
    if (k + 1 < M.nlev) {
        const size_t o = (size_t)(k + 1) * ncol + c;
        v += LUMP ? __ldg(uv + o) * __ldg(M.rmlump + o) : __ldg(uv + o);
    }
    if (k > 0) {
        const size_t o = (size_t)k * ncol + c;
        v -= LUMP ? __ldg(uv + o) * __ldg(M.rmlump + o) : __ldg(uv + o);
    }
    return s + __ldg(M.divv + k) * v;
}

// velocity rows on horizontal faces: yh = M_h uh + kd (p_R - p_L)          [MODE 0]
// Step 3 on horizontal faces:         yh = (uh - kd (p_R - p_L)) / m_h    [MODE 1, times 1 / m_h]
// rows of A-hat:                      yh = (W^-1 M_h^T W uh) + kd (p_R - p_L)  [MODE 2]
template <int MODE>
__global__ void k_mx_faces_h(MixedDev M, const double* __restrict__ uh, const double* __restrict__ p,
                             double* __restrict__ yh) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (f >= M.nfh) return;
    const size_t o = (size_t)k * M.nfh + f, op = (size_t)k * M.ncol;
    const double g = __ldg(M.kd_h + o) * (__ldg(p + op + __ldg(M.faceR + f)) - __ldg(p + op + __ldg(M.faceL + f)));
    if (MODE == 0) {
        double m = M.ms * __ldg(uh + o);
        const double* ul = uh + (size_t)k * M.nfh;
        for (int t = 0; t < M.ncf; ++t)
            m += __ldg(M.wf + (size_t)t * M.nfh + f) * __ldg(ul + __ldg(M.cf + (size_t)t * M.nfh + f));
        yh[o] = m + g;
    } else if (MODE == 2) {
        const double* ul = uh + (size_t)k * M.nfh;
        const double* Wl = M.Wf + (size_t)k * M.nfh;
        double m = 0.0;
        for (int t = 0; t < M.ncf; ++t) {
            const int gf = __ldg(M.cf + (size_t)t * M.nfh + f);
            m += __ldg(M.wfT + (size_t)t * M.nfh + f) * (__ldg(Wl + gf) * __ldg(ul + gf));
        }
        yh[o] = (M.ms * __ldg(uh + o) + m / __ldg(Wl + f)) + g;
    } else {
        yh[o] = (__ldg(uh + o) - g) * __ldg(M.rmlump_h + f);
    }
}

// velocity rows on vertical faces: yv = M-bar uv + kd (p_kf - p_kf-1)   [MODE 0]
// rows of A-hat: the couplings of M-bar^T (face kf+1's coupling down, face kf-1's up)
// weighted by W_neighbour / W_kf                                        [MODE 2]
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
        yv[o] = M.mv * __ldg(uv + o) + __ldg(M.w_up + o) * __ldg(uv + o + ncol) + __ldg(M.w_dn + o) * __ldg(uv + o - ncol) + g;
    } else if (MODE == 2) {
        const double* Wv = M.Wf + (size_t)M.nlev * M.nfh;
        const double m = __ldg(M.w_dn + o + ncol) * (__ldg(Wv + o + ncol) * __ldg(uv + o + ncol)) +
                         __ldg(M.w_up + o - ncol) * (__ldg(Wv + o - ncol) * __ldg(uv + o - ncol));
        yv[o] = (M.mv * __ldg(uv + o) + m / __ldg(Wv + o)) + g;
    } else {
        yv[o] = (__ldg(uv + o) - g) * __ldg(M.rmlump + o);
    }
}

// [out_u; out_p] = J S^-1 [in_u; in_p] (MULT false) or S J [in_u; in_p] (MULT true), with
// S = diag(W, V) (V = area dz, the cell volumes) and J = diag(I, -I)
template <bool MULT>
__global__ void k_mx_adj_scale(MixedDev M, size_t nu, const double* __restrict__ area, const double* __restrict__ dz,
                               const double* in_u, const double* in_p, double* out_u, double* out_p) {
    const size_t np = (size_t)M.nlev * M.ncol;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nu + np; i += (size_t)gridDim.x * blockDim.x) {
        if (i < nu) {
            const double w = __ldg(M.Wf + i);
            out_u[i] = MULT ? in_u[i] * w : in_u[i] / w;
        } else {
            const size_t e = i - nu;
            const int k = (int)(e / M.ncol), c = (int)(e - (size_t)k * M.ncol);
            const double v = __ldg(area + c) * __ldg(dz + k);
            out_p[e] = MULT ? -(in_p[e] * v) : -(in_p[e] / v);
        }
    }
}

// dL/dg_i = -sum over the faces f of cell i of lam_f (p_R(f) - p_L(f)) c_s dt / (2 d_f): the
// background factors enter the mixed operator only through the gradient weights
// kappa_f / d_f = c_s dt (g_i + g_j) / (2 d_f).  One thread per cell.
__global__ void k_mx_grad_g(MixedDev M, const double* __restrict__ lam_u, const double* __restrict__ p,
                            double* __restrict__ grad_g) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (c >= M.ncol) return;
    const size_t ncol = M.ncol, op = (size_t)k * ncol;
    const double* lh = lam_u + (size_t)k * M.nfh;
    const double* lv = lam_u + (size_t)M.nlev * M.nfh;
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int f = __ldg(M.fof + d * ncol + c);
        s -= lh[f] * (__ldg(p + op + __ldg(M.faceR + f)) - __ldg(p + op + __ldg(M.faceL + f))) * __ldg(M.cdh + f);
    }
    if (k >= 1)   // face k below the cell
        s -= lv[op + c] * (__ldg(p + op + c) - __ldg(p + op - ncol + c)) * __ldg(M.cdv + k);
    if (k + 1 <= M.nlev - 1)   // face k + 1 above it
        s -= lv[op + ncol + c] * (__ldg(p + op + ncol + c) - __ldg(p + op + c)) * __ldg(M.cdv + k + 1);
    grad_g[op + c] = s;
}

// dL/dbeta_up[kf] = -eps lam_kf u_kf+1 and dL/dbeta_dn[kf] = -eps lam_kf u_kf-1 on the
// vertical faces whose coupling exists (both faces interior), 0 elsewhere.
__global__ void k_mx_grad_beta(MixedDev M, const double* __restrict__ lam_v, const double* __restrict__ uv,
                               double* __restrict__ gup, double* __restrict__ gdn) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, kf = blockIdx.y;
    if (c >= M.ncol) return;
    const size_t ncol = M.ncol, o = (size_t)kf * ncol + c;
    const int nlev = M.nlev;
    gup[o] = (kf >= 1 && kf + 1 <= nlev - 1) ? -M.eps * lam_v[o] * uv[o + ncol] : 0.0;
    gdn[o] = (kf >= 2 && kf <= nlev - 1) ? -M.eps * lam_v[o] * uv[o - ncol] : 0.0;
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

// Pressure-system GCR pass 1: w = H z (FP64, Eq. helmholtz_operator) for the levels
// [k0, k0 + kchunk) of one column per thread, fused with the GCR sums of the new direction J.
// The finest level keeps its six couplings per cell premultiplied in FP64 (a6[side][k][c],
// sides E, W, N, S, up, down), so H z costs 6 differences and 6 fused multiply-adds: FP64
// issue, not memory, bounds this kernel on GB300.
template <int J>
__global__ void __launch_bounds__(RED_THREADS) k_apply_gcr(Lvl<double, double> L, const double* __restrict__ a6,
                                                           const double* __restrict__ z, double* __restrict__ w,
                                                           const double* __restrict__ Wb, size_t ld,
                                                           const double* __restrict__ r, int kchunk,
                                                           double* partials, unsigned int* ticket, GcrScal* S) {
    double v[J + 2], t[J + 2];
#pragma unroll
    for (int i = 0; i < J + 2; ++i) v[i] = 0.0;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < L.ncol) {
        const size_t ncol = L.ncol, N = (size_t)L.nlev * ncol;
        const int k0 = blockIdx.y * kchunk;
        const int k1 = min(L.nlev, k0 + kchunk);
        int nb[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) nb[s] = __ldg(L.nbr + s * ncol + c);
        double xm = k0 > 0 ? __ldg(z + (size_t)(k0 - 1) * ncol + c) : 0.0;
        double x0 = __ldg(z + (size_t)k0 * ncol + c);
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const size_t o = (size_t)k * ncol, e = o + c;
            const double xp = (k + 1 < L.nlev) ? __ldg(z + o + ncol + c) : 0.0;
#if MG_APPLY_DIAG
            // diagonal form: (1 + sum_f a_f) x_i - sum_f a_f x_j, 7 FP64 operations
            double we = __ldg(a6 + 6 * N + e) * x0;
            we = fma(-__ldg(a6 + e), __ldg(z + o + nb[0]), we);
            we = fma(-__ldg(a6 + N + e), __ldg(z + o + nb[1]), we);
            we = fma(-__ldg(a6 + 2 * N + e), __ldg(z + o + nb[2]), we);
            we = fma(-__ldg(a6 + 3 * N + e), __ldg(z + o + nb[3]), we);
            we = fma(-__ldg(a6 + 4 * N + e), xp, we);
            we = fma(-__ldg(a6 + 5 * N + e), xm, we);
#else
            double we = x0;
            we = fma(__ldg(a6 + e), x0 - __ldg(z + o + nb[0]), we);
            we = fma(__ldg(a6 + N + e), x0 - __ldg(z + o + nb[1]), we);
            we = fma(__ldg(a6 + 2 * N + e), x0 - __ldg(z + o + nb[2]), we);
            we = fma(__ldg(a6 + 3 * N + e), x0 - __ldg(z + o + nb[3]), we);
            we = fma(__ldg(a6 + 4 * N + e), x0 - xp, we);
            we = fma(__ldg(a6 + 5 * N + e), x0 - xm, we);
#endif
            w[e] = we;
            gcr_accumulate<J>(v, we, __ldg(r + e), Wb, ld, e);
            xm = x0;
            x0 = xp;
        }
    }
    if (grid_reduce<J + 2>(v, partials, ticket, t)) gcr_coeffs<J>(t, S);
}

}  // namespace mg
