// C ABI of the GB300 column multigrid solver: handle, set-up, V-cycle driver (Algorithm 1),
// GCR outer solves and the mixed-system Schur-complement preconditioner.
// See include/mgsolve.h for the contract of every entry point.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/mgsolve.h"
#include "kernels.cuh"
#include "krylov.cuh"
#include "mesh.h"

// tuning knobs of the sweep kernel (FP32 prefetch depths, threads per block)
#ifndef MG_SWEEP_DEEP32
#define MG_SWEEP_DEEP32 4
#endif
#ifndef MG_SWEEP_SHAL32
#define MG_SWEEP_SHAL32 4
#endif
// residual + restriction on levels with n % 16 == 0: levels per thread, levels loaded ahead
#ifndef MG_RESTRICT_KCHUNK
#define MG_RESTRICT_KCHUNK 8
#endif
#ifndef MG_RESTRICT_KCHUNK_BIG
#define MG_RESTRICT_KCHUNK_BIG 24
#endif
#ifndef MG_RESTRICT_BIG_NCOL
#define MG_RESTRICT_BIG_NCOL 100000
#endif
#ifndef MG_RESTRICT_ASYNC
#define MG_RESTRICT_ASYNC 1          // FP32 levels: own-column streams through a copy ring
#endif
#ifndef MG_RESTRICT_ASYNC_NCOL
#define MG_RESTRICT_ASYNC_NCOL 40000 // smaller levels: the register ring alone is as fast
#endif
#ifndef MG_RESTRICT_DEEP
#define MG_RESTRICT_DEEP 4
#endif
#ifndef MG_RESTRICT_ASHAL
#define MG_RESTRICT_ASHAL 2
#endif
#ifndef MG_RESTRICT_SHAL
#define MG_RESTRICT_SHAL 2
#endif
#ifndef MG_SWEEP_SHAL_PRO
#define MG_SWEEP_SHAL_PRO 2
#endif
#ifndef MG_SWEEP_SHAL_ZERO
#define MG_SWEEP_SHAL_ZERO 2
#endif
#ifndef MG_SWEEP_BLOCK
#define MG_SWEEP_BLOCK 128
#endif

using mg::Lvl;
typedef __nv_bfloat16 bf16;

namespace {

struct DevLevel {
    int n = 0, ncol = 0;
    int32_t* nbr = nullptr;
    int32_t* fof = nullptr;
    double* rA64 = nullptr;
    float* rA32 = nullptr;
    double* Th64 = nullptr;
    double* Tv64 = nullptr;
    float* Th32 = nullptr;
    float* Tv32 = nullptr;
    bf16* Th16 = nullptr;
    bf16* Tv16 = nullptr;
    double* w64 = nullptr;  // restriction weights onto the next level, [4][ncol_next]
    float* w32 = nullptr;
    // workspace: two iterates, the level's rhs and the result handed to the finer level
    double* x64[2] = {nullptr, nullptr};
    double* b64 = nullptr;
    double* r64 = nullptr;
    float* x32[2] = {nullptr, nullptr};
    float* b32 = nullptr;
    float* r32 = nullptr;
    // launch shapes chosen by mg_autotune (0 / -1: the built-in choice)
    int sweep_bd = 0;          // threads per sweep block, a multiple of 64
    int restrict_kc = 0;       // levels per thread of the residual + restriction
    int restrict_async = -1;   // 1: copy-ring restriction (FP32 levels, n % 16 = 0), 0: register ring
    // 9-cell stencil: fluxes two levels apart [nlev][ncol] and three scratch fields (the
    // residual and the two Thomas factors of a sweep)
    double* T2_64 = nullptr;
    float* T2_32 = nullptr;
    double* s64[3] = {nullptr, nullptr, nullptr};
    float* s32[3] = {nullptr, nullptr, nullptr};
};

}  // namespace

struct mg_handle {
    int device = 0;
    int L = 0, nlev = 0, n = 0;
    int nsm = 0;
    mg_params prm{};
    std::vector<DevLevel> lv;
    double* rdz64 = nullptr;
    float* rdz32 = nullptr;
    double* a6 = nullptr;       // finest level: six premultiplied FP64 couplings and 1 + their sum, per cell
    bool nine = false;          // 9-cell stencil (mg_setup_9pt)
    bool pivot64 = false;       // MG_FP32_P64: FP64 elimination in the finest level's FP32 sweeps
    double* area0 = nullptr;    // finest level: column areas and layer depths (cell volumes, adjoint solve)
    double* dz = nullptr;
    double* adj = nullptr;      // [N] the scaled right-hand side of the adjoint solve
    // finest-level face tables for caller-supplied couplings (mg_setup_coeffs, mg_set_coefficients)
    int32_t* faceL0 = nullptr;
    int32_t* faceR0 = nullptr;
    int32_t* faceSide0 = nullptr;
    int32_t* nbrSide0 = nullptr;
    unsigned int* flag = nullptr;
    // pressure solver K_H(A_H, P_H, eps_H) of the Schur-complement step (Sec. 4.1, Table 1)
    mg_pressure_solver ps{MG_PS_MG, 1e-2, 0.8, 10, 200};
    double* bv[8] = {};             // BiCGStab vectors r^, r, p, v, s, t, p^, s^ (allocated on demand)
    mg::BicgScal* bs = nullptr;     // its device scalars
    mg::BicgScal* host_bs = nullptr;   // pinned copy read once per iteration
    long long ps_solves = 0;        // pressure solves since the last mg_inner_stats
    double ps_iters = 0.0;          // their BiCGStab iterations (a half step counts 0.5)
    // GCR
    size_t glen = 0;            // length of a GCR vector (N, or nu + N with mixed data)
    double* Z = nullptr;        // [restart][glen]
    double* W = nullptr;        // [restart][glen]
    double* r = nullptr;        // [glen]
    mg::GcrScal* gs = nullptr;  // device scalars of the GCR iteration
    double* partials = nullptr;
    size_t npartials = 0;
    unsigned int* tickets = nullptr;
    double* host_sc = nullptr;  // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // one CUDA graph per GCR slot j and system (0 pressure, 1 mixed, 2 the mixed adjoint's
    // A-hat): the V-cycle, the
    // operator with its sums, the orthogonalisation and the read-back of <r, r>, captured on
    // `cap` the first time and replayed on the caller's stream afterwards
    cudaStream_t cap = nullptr;
    cudaStream_t run = nullptr;   // the handle's stream inside an ensemble solve
    cudaEvent_t evx = nullptr;    // ordering event (no timing)
    cudaGraphExec_t gexec[3][mg::MAXR] = {};
    bool graphs_off = false;
    int red_grid = 0;
    // mixed
    bool mixed = false;
    int64_t nu = 0;
    mg::MixedDev md{};
    double* schurB = nullptr;
    double* mb = nullptr;       // concatenated mixed rhs [nu + N]
    double* mx = nullptr;       // concatenated mixed solution [nu + N]
    std::vector<void*> allocs;
    // per-launch event profiling (mg_profile_start / mg_profile_stop)
    struct Rec {
        int kind, level, variant;
        double bytes;
    };
    bool prof = false;
    int prof_kind = -1, prof_level = -1;   // record only this kind / level (-1: all)
    std::vector<cudaEvent_t> evpool;
    std::vector<Rec> recs;
};

namespace {

enum { TK_DOT = 0, TK_SUMS, TK_ORTH, TK_BICG, TK_COUNT };

// k-chunk of the column kernels that have no vertical recurrence (apply): short chunks give
// many independent threads, so the loads of different threads overlap
constexpr int APPLY_KCHUNK = 8;

// the CUDA error behind the last MG_ERR_CUDA of this thread (mg_last_cuda_error)
thread_local cudaError_t g_last_cuda = cudaSuccess;

// A failed runtime call returns MG_ERR_CUDA; a non-sticky error is cleared so that it does not
// surface again in a later, unrelated call.
#define CK(call)                       \
    do {                               \
        cudaError_t e_ = (call);       \
        if (e_ != cudaSuccess) {       \
            g_last_cuda = e_;          \
            cudaGetLastError();        \
            return MG_ERR_CUDA;        \
        }                              \
    } while (0)

// Every device and pinned-host allocation of the library goes through mem_alloc / mem_free.
// They count the live allocations (mg_live_allocations) and carry the failure injection of
// mg_inject_alloc_failure: with g_fail_at = n > 0, the n-th allocation attempted after the call
// fails as if the memory were exhausted.
std::atomic<long long> g_fail_at{0}, g_alloc_seen{0}, g_live{0};

enum MemKind { MEM_DEVICE, MEM_PINNED };

bool mem_alloc(void** p, size_t bytes, MemKind kind) {
    *p = nullptr;
    const long long seen = g_alloc_seen.fetch_add(1) + 1;
    const long long at = g_fail_at.load();
    if (at > 0 && seen == at) return false;
    const cudaError_t e = kind == MEM_DEVICE ? cudaMalloc(p, bytes) : cudaMallocHost(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    g_live.fetch_add(1);
    return true;
}

void mem_free(void* p, MemKind kind) {
    if (!p) return;
    if (kind == MEM_DEVICE) cudaFree(p);
    else cudaFreeHost(p);
    g_live.fetch_sub(1);
}

template <typename P>
mg_status dalloc(mg_handle* h, P** p, size_t count) {
    *p = nullptr;
    if (count == 0) return MG_OK;
    void* q = nullptr;
    if (!mem_alloc(&q, count * sizeof(P), MEM_DEVICE)) return MG_ERR_NOMEM;
    h->allocs.push_back(q);
    *p = static_cast<P*>(q);
    return MG_OK;
}

template <typename P, typename S>
mg_status upload(mg_handle* h, P** p, const std::vector<S>& src) {
    mg_status st = dalloc(h, p, src.size());
    if (st != MG_OK) return st;
    if (src.empty()) return MG_OK;
    std::vector<P> tmp(src.size());
    for (size_t i = 0; i < src.size(); ++i) tmp[i] = (P)src[i];
    CK(cudaMemcpy(*p, tmp.data(), tmp.size() * sizeof(P), cudaMemcpyHostToDevice));
    return MG_OK;
}

template <>
mg_status upload<bf16, double>(mg_handle* h, bf16** p, const std::vector<double>& src) {
    mg_status st = dalloc(h, p, src.size());
    if (st != MG_OK) return st;
    std::vector<bf16> tmp(src.size());
    for (size_t i = 0; i < src.size(); ++i) tmp[i] = __float2bfloat16_rn((float)src[i]);
    CK(cudaMemcpy(*p, tmp.data(), tmp.size() * sizeof(bf16), cudaMemcpyHostToDevice));
    return MG_OK;
}

// An NVTX range over the scope (shows the library's calls and GCR iterations on a profiler's
// timeline; costs nothing without a tool attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

#define TRY(call)                         \
    do {                                  \
        mg_status s_ = (call);            \
        if (s_ != MG_OK) return s_;       \
    } while (0)

inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

inline size_t cells(const mg_handle* h, int l) { return (size_t)h->nlev * h->lv[l].ncol; }

// Brackets one kernel launch with a pair of events when profiling is on.  `bytes` is the
// algorithmic traffic of the launch: every array element the kernel must read or write,
// counted once (neighbour re-reads within a launch are cache traffic, not counted).
struct Prof {
    mg_handle* h;
    cudaStream_t s;
    int idx = -1;
    Prof(mg_handle* h_, int kind, int level, double bytes, cudaStream_t s_, int variant = 0) : h(h_), s(s_) {
        if (h && h->prof && 2 * (h->recs.size() + 1) <= h->evpool.size() &&
            (h->prof_kind < 0 || h->prof_kind == kind) && (h->prof_level < 0 || h->prof_level == level)) {
            idx = (int)h->recs.size();
            h->recs.push_back({kind, level, variant, bytes});
            cudaEventRecord(h->evpool[2 * idx], s);
        }
    }
    ~Prof() {
        if (idx >= 0) cudaEventRecord(h->evpool[2 * idx + 1], s);
    }
};

// ---- per-precision views of a level ----
template <typename T, typename C>
struct View;

template <>
struct View<double, double> {
    static Lvl<double, double> lvl(const mg_handle* h, int l) {
        const DevLevel& d = h->lv[l];
        return {d.n, d.ncol, h->nlev, d.nbr, d.fof, d.Th64, d.Tv64, d.rA64, h->rdz64};
    }
    static double* x(DevLevel& d, int i) { return d.x64[i]; }
    static double* b(DevLevel& d) { return d.b64; }
    static double* r(DevLevel& d) { return d.r64; }
    static const double* w(const DevLevel& d) { return d.w64; }
    static const double* t2(const DevLevel& d) { return d.T2_64; }
    static double* scratch(DevLevel& d, int i) { return d.s64[i]; }
};
template <>
struct View<float, float> {
    static Lvl<float, float> lvl(const mg_handle* h, int l) {
        const DevLevel& d = h->lv[l];
        return {d.n, d.ncol, h->nlev, d.nbr, d.fof, d.Th32, d.Tv32, d.rA32, h->rdz32};
    }
    static float* x(DevLevel& d, int i) { return d.x32[i]; }
    static float* b(DevLevel& d) { return d.b32; }
    static float* r(DevLevel& d) { return d.r32; }
    static const float* w(const DevLevel& d) { return d.w32; }
    static const float* t2(const DevLevel& d) { return d.T2_32; }
    static float* scratch(DevLevel& d, int i) { return d.s32[i]; }
};
template <>
struct View<float, bf16> {
    static Lvl<float, bf16> lvl(const mg_handle* h, int l) {
        const DevLevel& d = h->lv[l];
        return {d.n, d.ncol, h->nlev, d.nbr, d.fof, d.Th16, d.Tv16, d.rA32, h->rdz32};
    }
    static float* x(DevLevel& d, int i) { return d.x32[i]; }
    static float* b(DevLevel& d) { return d.b32; }
    static float* r(DevLevel& d) { return d.r32; }
    static const float* w(const DevLevel& d) { return d.w32; }
};

constexpr size_t SWEEP_SMEM_MAX = 200 * 1024;

inline int sweep_block(int ncol) {
    if (ncol >= 128 * 300) return MG_SWEEP_BLOCK;
    if (ncol >= 64 * 300) return 64;
    return 32;
}

// ---- launchers ----
template <typename T, typename C, typename X, typename Y>
mg_status launch_apply(mg_handle* h, int lev, const Lvl<T, C>& L, const X* x, Y* y, cudaStream_t s) {
    const double nc = (double)L.nlev * L.ncol;
    Prof pr(h, MG_K_APPLY, lev, nc * (sizeof(X) + 3 * sizeof(C) + sizeof(Y)), s);
    const int bd = 128;
    const int kc = APPLY_KCHUNK;
    dim3 grid((L.ncol + bd - 1) / bd, (L.nlev + kc - 1) / kc);
    mg::k_apply<T, C, X, Y><<<grid, bd, 0, s>>>(L, x, y, kc);
    CK(cudaGetLastError());
    return MG_OK;
}

// prefetch depths of the sweep's register rings (levels in flight per thread)
template <typename T>
struct SweepPF {
    static constexpr int deep = sizeof(T) == 8 ? 4 : MG_SWEEP_DEEP32;
    static constexpr int shal = sizeof(T) == 8 ? 2 : MG_SWEEP_SHAL32;
};

// FP32 levels of 30, 50 or 70 levels use the register-stash sweep (k_sweep_rs) where it was
// measured faster at C192L70: every sweep from a zero iterate (the first of each level; finest
// level 107 us against 110, levels 1-3 27 / 14 / 11 us against 36 / 20 / 19), and the plain
// sweeps of levels of at most MG_SWEEP_RS_PLAIN_NCOL columns (the coarsest, 13 us against 15).
// On larger levels its eleven staged words per step make the plain sweep slower (167 us against
// 121 on the finest level), and the sweep with fused prolongation slower on every level.
#ifndef MG_SWEEP_REG
#define MG_SWEEP_REG 1
#endif
#ifndef MG_SWEEP_RS_PLAIN_NCOL
#define MG_SWEEP_RS_PLAIN_NCOL 4000
#endif

// The register-stash sweep (k_sweep_rs) for an FP32 level of NLEV levels, bd threads per block
template <int NLEV, int MODE, typename B, typename O, bool BCOPY>
mg_status launch_sweep_rs(const Lvl<float, float>& L, const float* x, const float* xc, int ncol_c, const B* b,
                          float* bcopy, O* xo, float omega, int bd, cudaStream_t s) {
    constexpr bool PRO = (MODE == mg::XM_PROLONG || MODE == mg::XM_PROLONG0);
    constexpr bool RAW = (MODE == mg::XM_PLAIN || MODE == mg::XM_PROLONG);
    // ring depth: the shared memory of the resident blocks (3 at 70 levels, else 4)
    constexpr int DEEP = mg::SweepRsBlocks<NLEV>::value == 3 ? ((PRO && RAW) ? 8 : 12) : ((PRO && RAW) ? 6 : 8);
    constexpr int NW = 5 + (RAW ? 5 : 0) + (PRO ? 5 : 0) + (sizeof(B) == 8 ? 0 : 1);
    const size_t smem = (size_t)DEEP * bd * (sizeof(B) == 8 ? 8 : 0) + (size_t)DEEP * NW * bd * 4 + NLEV * 4;
    auto kern = mg::k_sweep_rs<NLEV, MODE, B, O, BCOPY, DEEP>;
    if (smem > 48 * 1024) CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (L.ncol + bd / 2 - 1) / (bd / 2);
    kern<<<grid, bd, smem, s>>>(L, x, xc, ncol_c, b, bcopy, xo, omega);
    CK(cudaGetLastError());
    return MG_OK;
}

template <typename T, typename C, int MODE, typename X, typename B, typename O, bool BCOPY, typename P>
mg_status launch_sweep_shared(mg_handle* h, int lev, const Lvl<T, C>& L, const X* x, const T* xc, int ncol_c,
                              const B* b, T* bcopy, O* xo, double omega, cudaStream_t s);

template <typename T, typename C, int MODE, typename X, typename B, typename O, bool BCOPY>
mg_status launch_sweep(mg_handle* h, int lev, const Lvl<T, C>& L, const X* x, const T* xc, int ncol_c,
                       const B* b, T* bcopy, O* xo, double omega, cudaStream_t s) {
    const double nc = (double)L.nlev * L.ncol;
    double per = sizeof(B) + 3 * sizeof(C) + sizeof(O);
    if (MODE == mg::XM_PLAIN || MODE == mg::XM_PROLONG) per += sizeof(X);
    if (MODE == mg::XM_PROLONG || MODE == mg::XM_PROLONG0) per += 0.25 * sizeof(T);
    if (BCOPY) per += sizeof(T);
    Prof pr(h, MG_K_SWEEP, lev, nc * per, s, MODE);
    if constexpr (std::is_same<T, float>::value && std::is_same<C, float>::value) {
        // MG_FP32_P64: the finest level eliminates with FP64 pivots
        if (h && h->pivot64 && lev == 0)
            return launch_sweep_shared<T, C, MODE, X, B, O, BCOPY, double>(h, lev, L, x, xc, ncol_c, b, bcopy, xo,
                                                                          omega, s);
    }
    if constexpr (MG_SWEEP_REG && std::is_same<T, float>::value && std::is_same<C, float>::value &&
                  std::is_same<X, float>::value && (MODE == mg::XM_ZERO || MODE == mg::XM_PLAIN)) {
        const int bdr = (h && h->lv[lev].sweep_bd > 0) ? h->lv[lev].sweep_bd : MG_SWEEP_BLOCK;
        const bool use = MODE == mg::XM_ZERO || L.ncol <= MG_SWEEP_RS_PLAIN_NCOL;
        if (use) switch (L.nlev) {
            case 70: return launch_sweep_rs<70, MODE, B, O, BCOPY>(L, x, xc, ncol_c, b, bcopy, xo, (float)omega, bdr, s);
            case 50: return launch_sweep_rs<50, MODE, B, O, BCOPY>(L, x, xc, ncol_c, b, bcopy, xo, (float)omega, bdr, s);
            case 30: return launch_sweep_rs<30, MODE, B, O, BCOPY>(L, x, xc, ncol_c, b, bcopy, xo, (float)omega, bdr, s);
            default: break;
        }
    }
    return launch_sweep_shared<T, C, MODE, X, B, O, BCOPY, T>(h, lev, L, x, xc, ncol_c, b, bcopy, xo, omega, s);
}

// the shared-memory-stash sweep (k_sweep), elimination in P
template <typename T, typename C, int MODE, typename X, typename B, typename O, bool BCOPY, typename P>
mg_status launch_sweep_shared(mg_handle* h, int lev, const Lvl<T, C>& L, const X* x, const T* xc, int ncol_c,
                              const B* b, T* bcopy, O* xo, double omega, cudaStream_t s) {
    // two threads per column; per thread the shared memory holds the asynchronous-copy
    // ring (DEEP slots of b, the next iterate and, unless BF16, three coefficients) and the
    // stash (2 values per step of half a column); it must fit the budget
    constexpr int DEEP = SweepPF<T>::deep;
    const int hsteps = (L.nlev + 1) / 2;
    // (BF16 coefficients travel as 4-byte pairs)
    const size_t per_thread =
        DEEP * (sizeof(B) + sizeof(T) + (sizeof(C) >= 4 ? 3 * sizeof(C) : (MG_SWEEP_BF16_PAIRS ? 12 : 0))) +
        2 * (size_t)hsteps * sizeof(T);
    const size_t per_block = (size_t)L.nlev * sizeof(T);   // the 1/dz table
    // (h is NULL for the allocation-free smoothing: built-in shapes)
    int bd = (h && h->lv[lev].sweep_bd > 0) ? h->lv[lev].sweep_bd : sweep_block(2 * L.ncol);
#if MG_SWEEP_WARP_HALVES
    constexpr int BQ = 64;   // the halves of a column lie in different warps
#else
    constexpr int BQ = 32;
#endif
    const int cap = (int)((SWEEP_SMEM_MAX - per_block) / per_thread) / BQ * BQ;
    if (cap < BQ) return MG_ERR_UNSUPPORTED;
    if (bd < BQ) bd = BQ;
    if (bd > cap) bd = cap;
    const size_t smem = per_thread * bd + per_block;
    // ring lengths per iterate source (measured at C192L70): a prolongation sweep with a fine
    // iterate carries eight neighbour values per step and needs the shorter ring to fit the
    // register budget; the zero-start sweep is fastest with the shorter ring as well
    constexpr int SHAL = MODE == mg::XM_PROLONG ? MG_SWEEP_SHAL_PRO
                         : MODE == mg::XM_ZERO    ? (sizeof(T) == 8 ? 2 : MG_SWEEP_SHAL_ZERO)
                                                  : SweepPF<T>::shal;
    auto kern = mg::k_sweep<T, C, MODE, X, B, O, BCOPY, DEEP, SHAL, P>;
    if (smem > 48 * 1024) CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int cols = bd / 2;
    const int grid = (L.ncol + cols - 1) / cols;
    kern<<<grid, bd, smem, s>>>(L, x, xc, ncol_c, b, bcopy, xo, (T)omega);
    CK(cudaGetLastError());
    return MG_OK;
}

template <typename T, typename C, bool XZERO, typename X, typename B, typename O>
mg_status launch_restrict(mg_handle* h, int lev, const Lvl<T, C>& L, const X* x, const B* b, const T* w, O* bc,
                          int ncol_c, cudaStream_t s) {
    const double nc = (double)L.nlev * L.ncol;
    Prof pr(h, MG_K_RESTRICT, lev, nc * (sizeof(B) + 3 * sizeof(C) + (XZERO ? 0 : sizeof(X)) + 0.25 * sizeof(O) +
                                          sizeof(T) / (double)L.nlev), s);
    if (L.n % 16 == 0) {
        // one thread per fine column, 4 warps per block
        const int warps = 6 * (L.n / 2) * (L.n / 16);
        // levels per thread: on a level large enough to fill the GPU several times over, long
        // chunks (fewer prologues); smaller levels need the threads of short chunks
        const int kc = (h && h->lv[lev].restrict_kc > 0) ? h->lv[lev].restrict_kc
                       : L.ncol >= MG_RESTRICT_BIG_NCOL ? MG_RESTRICT_KCHUNK_BIG
                                                        : MG_RESTRICT_KCHUNK;
        const dim3 grid((warps + 3) / 4, (L.nlev + kc - 1) / kc);
        constexpr bool ASYNC = MG_RESTRICT_ASYNC && !XZERO && std::is_same<T, float>::value &&
                               std::is_same<C, float>::value && std::is_same<X, float>::value &&
                               std::is_same<B, float>::value && std::is_same<O, float>::value;
        bool async_done = false;
        if constexpr (ASYNC) {
            const int ra = h ? h->lv[lev].restrict_async : -1;
            if (ra >= 0 ? ra == 1 : L.ncol >= MG_RESTRICT_ASYNC_NCOL) {
                mg::k_resid_restrict16a<MG_RESTRICT_DEEP, MG_RESTRICT_ASHAL><<<grid, 128, 0, s>>>(L, x, b, w, bc,
                                                                                                 ncol_c, kc);
                async_done = true;
            }
        }
        if (!async_done)
            mg::k_resid_restrict16<T, C, XZERO, X, B, O, MG_RESTRICT_SHAL><<<grid, 128, 0, s>>>(L, x, b, w, bc,
                                                                                               ncol_c, kc);
        CK(cudaGetLastError());
        return MG_OK;
    }
    const int bd = ncol_c >= 128 * 300 ? 128 : (ncol_c >= 64 * 300 ? 64 : 32);
    // chunk of levels per thread: enough threads to fill the GPU, few re-loads of the
    // 32 connectivity entries of the 4 children
    const int kc = (h && h->lv[lev].restrict_kc > 0) ? h->lv[lev].restrict_kc
                   : ncol_c >= 128 * 300 ? 3 * APPLY_KCHUNK
                                         : APPLY_KCHUNK;
    const dim3 grid((ncol_c + bd - 1) / bd, (L.nlev + kc - 1) / kc);
    mg::k_resid_restrict<T, C, XZERO, X, B, O><<<grid, bd, 0, s>>>(L, x, b, w, bc, ncol_c, kc);
    CK(cudaGetLastError());
    return MG_OK;
}

template <typename T, bool ZB, typename X, typename O>
mg_status launch_prolong(mg_handle* h, int lev, int n, int ncol, int ncol_c, int nlev, const X* x, const T* xc,
                         O* xo, cudaStream_t s) {
    Prof pr(h, MG_K_PROLONG, lev, (double)nlev * ncol * (0.25 * sizeof(T) + (ZB ? 0 : sizeof(X)) + sizeof(O)), s);
    const int bd = 128;
    mg::k_prolong<T, ZB, X, O><<<(ncol + bd - 1) / bd, bd, 0, s>>>(n, ncol, ncol_c, nlev, x, xc, xo);
    CK(cudaGetLastError());
    return MG_OK;
}

template <typename A, typename B>
mg_status launch_convert(mg_handle* h, int lev, size_t n, const A* a, B* b, cudaStream_t s) {
    Prof pr(h, MG_K_CONVERT, lev, (double)n * (sizeof(A) + sizeof(B)), s);
    mg::k_convert<A, B><<<4 * 152, 256, 0, s>>>(n, a, b);
    CK(cudaGetLastError());
    return MG_OK;
}

// One sweep with the iterate source chosen at run time.
//   cur == nullptr and xc == nullptr : zero iterate
//   xc != nullptr                    : iterate = (cur or 0) + Prolongate(xc)
template <typename T, typename C, typename B, typename O>
mg_status sweep_any(mg_handle* h, int lev, const Lvl<T, C>& L, const T* cur, const T* xc, int ncol_c, const B* b,
                    T* bcopy, O* xo, double om, cudaStream_t s) {
    if (bcopy) {
        if (xc) return MG_ERR_ARG;
        if (cur) return launch_sweep<T, C, mg::XM_PLAIN, T, B, O, true>(h, lev, L, cur, xc, ncol_c, b, bcopy, xo, om, s);
        return launch_sweep<T, C, mg::XM_ZERO, T, B, O, true>(h, lev, L, cur, xc, ncol_c, b, bcopy, xo, om, s);
    }
    if (xc) {
        if (cur)
            return launch_sweep<T, C, mg::XM_PROLONG, T, B, O, false>(h, lev, L, cur, xc, ncol_c, b, bcopy, xo, om, s);
        return launch_sweep<T, C, mg::XM_PROLONG0, T, B, O, false>(h, lev, L, cur, xc, ncol_c, b, bcopy, xo, om, s);
    }
    if (cur) return launch_sweep<T, C, mg::XM_PLAIN, T, B, O, false>(h, lev, L, cur, xc, ncol_c, b, bcopy, xo, om, s);
    return launch_sweep<T, C, mg::XM_ZERO, T, B, O, false>(h, lev, L, cur, xc, ncol_c, b, bcopy, xo, om, s);
}

// Settings of one cycle: levels used, over-relaxation and sweep counts.  A single-level
// cycle with n_coarse sweeps is the block-Jacobi iteration P_H^(Jac)(omega, n_coarse) of
// Sec. 4.1 (line relaxation).
struct Cycle {
    int L;
    double omega;
    int n_pre, n_post, n_coarse;
};

inline Cycle vcycle_of(const mg_handle* h) {
    return {h->L, h->prm.omega, h->prm.n_pre, h->prm.n_post, h->prm.n_coarse};
}

// Algorithm 1 on level l with right-hand side `b` (type B: FP64 on the finest level of the
// FP32 V-cycle, T otherwise); the result goes to `out` (type O).  On every level the
// iterate starts at zero (x^(l+1) <- 0 of Algorithm 1; the V-cycle is used as a
// preconditioner, so x^(1) = 0 as well).
template <typename T, typename C, typename B, typename O>
mg_status mgv(mg_handle* h, const Cycle& cy, int l, const B* b, O* out, cudaStream_t s) {
    static const char* const level_range[MG_MAX_LEVELS] = {"V-cycle level 0", "V-cycle level 1", "V-cycle level 2",
                                                           "V-cycle level 3", "V-cycle level 4", "V-cycle level 5",
                                                           "V-cycle level 6", "V-cycle level 7"};
    NvtxRange nvtx_(level_range[l]);   // the level and the levels below it (nested ranges)
    typedef View<T, C> V;
    DevLevel& d = h->lv[l];
    const Lvl<T, C> L = V::lvl(h, l);
    const bool coarsest = (l == cy.L - 1);
    const double om = cy.omega;
    const bool conv = !std::is_same<B, T>::value;  // rhs arrives in FP64, iterate in FP32
    T* ws[2] = {V::x(d, 0), V::x(d, 1)};
    const T* bT = conv ? (const T*)V::b(d) : (const T*)(const void*)b;
    const int npre = coarsest ? cy.n_coarse : cy.n_pre;
    if (conv && npre == 0) TRY(launch_convert(h, l, cells(h, l), b, V::b(d), s));
    T* cur = nullptr;
    for (int i = 0; i < npre; ++i) {
        const bool final = coarsest && i == npre - 1;
        T* dst = (cur == ws[0]) ? ws[1] : ws[0];
        T* bcopy = (conv && i == 0) ? V::b(d) : nullptr;
        if (final) {
            if (i == 0) TRY((sweep_any<T, C, B, O>(h, l, L, cur, (const T*)nullptr, 0, b, bcopy, out, om, s)));
            else TRY((sweep_any<T, C, T, O>(h, l, L, cur, (const T*)nullptr, 0, bT, nullptr, out, om, s)));
            return MG_OK;
        }
        if (i == 0) TRY((sweep_any<T, C, B, T>(h, l, L, cur, (const T*)nullptr, 0, b, bcopy, dst, om, s)));
        else TRY((sweep_any<T, C, T, T>(h, l, L, cur, (const T*)nullptr, 0, bT, nullptr, dst, om, s)));
        cur = dst;
    }
    // residual and restriction onto level l+1
    DevLevel& dc = h->lv[l + 1];
    T* bc = V::b(dc);
    if (cur) TRY((launch_restrict<T, C, false, T, T, T>(h, l, L, cur, bT, V::w(d), bc, dc.ncol, s)));
    else TRY((launch_restrict<T, C, true, T, T, T>(h, l, L, cur, bT, V::w(d), bc, dc.ncol, s)));
    T* xc = V::r(dc);
    TRY((mgv<T, C, T, T>(h, cy, l + 1, bc, xc, s)));
    // coarse-grid correction fused into the first post-smoothing sweep
    const int npost = cy.n_post;
    if (npost == 0) {
        if (cur) return launch_prolong<T, false, T, O>(h, l, d.n, d.ncol, dc.ncol, h->nlev, cur, xc, out, s);
        return launch_prolong<T, true, T, O>(h, l, d.n, d.ncol, dc.ncol, h->nlev, cur, xc, out, s);
    }
    for (int i = 0; i < npost; ++i) {
        const T* pxc = (i == 0) ? xc : nullptr;
        const int ncc = (i == 0) ? dc.ncol : 0;
        if (i == npost - 1) return sweep_any<T, C, T, O>(h, l, L, cur, pxc, ncc, bT, nullptr, out, om, s);
        T* dst = (cur == ws[0]) ? ws[1] : ws[0];
        TRY((sweep_any<T, C, T, T>(h, l, L, cur, pxc, ncc, bT, nullptr, dst, om, s)));
        cur = dst;
    }
    return MG_OK;
}

// ---- the 9-cell stencil (Sec. 3.5): V-cycle with the tridiagonal smoother H_z-hat ----
// x_out = x + omega Hz^-1 (b - H x), x == NULL meaning a zero iterate: the residual with the
// full 9-cell stencil, then the column solves without the next-to-nearest fluxes
template <typename T, typename B, typename O>
mg_status sweep9(mg_handle* h, int lev, const T* x, const B* b, O* xo, double omega, cudaStream_t s) {
    typedef View<T, T> V;
    DevLevel& d = h->lv[lev];
    const Lvl<T, T> L = V::lvl(h, lev);
    Prof pr(h, MG_K_SWEEP, lev, (double)L.nlev * L.ncol * (sizeof(B) + 4.0 * sizeof(T) + sizeof(O) +
                                                           (x ? 2.0 * sizeof(T) : 0.0)), s);
    const dim3 g2((L.ncol + 127) / 128, L.nlev);
    mg::k_resid9<T, B><<<g2, 128, 0, s>>>(L, V::t2(d), x, b, V::scratch(d, 0));
    mg::k_thomas9<T, O><<<(L.ncol + 127) / 128, 128, 0, s>>>(L, V::scratch(d, 0), x, V::scratch(d, 1),
                                                              V::scratch(d, 2), xo, (T)omega);
    CK(cudaGetLastError());
    return MG_OK;
}

// y = H x on level `lev` in FP64 for the 9-cell stencil
mg_status launch_apply9(mg_handle* h, int lev, const double* x, double* y, cudaStream_t s) {
    const Lvl<double, double> L = View<double, double>::lvl(h, lev);
    Prof pr(h, MG_K_APPLY, lev, (double)L.nlev * L.ncol * 8.0 * 6, s);
    mg::k_apply9<double, double, double><<<dim3((L.ncol + 127) / 128, L.nlev), 128, 0, s>>>(L, h->lv[lev].T2_64, x, y);
    CK(cudaGetLastError());
    return MG_OK;
}

// bc = Restrict(b - H x) onto level lev + 1 (9-cell stencil; x == NULL: zero iterate)
template <typename T, typename B, typename O>
mg_status restrict9(mg_handle* h, int lev, const T* x, const B* b, O* bc, cudaStream_t s) {
    typedef View<T, T> V;
    DevLevel& d = h->lv[lev];
    const DevLevel& dc = h->lv[lev + 1];
    const Lvl<T, T> L = V::lvl(h, lev);
    Prof pr(h, MG_K_RESTRICT, lev, (double)L.nlev * L.ncol * (sizeof(B) + 2.0 * sizeof(T) + 0.25 * sizeof(O)), s);
    const dim3 g2((L.ncol + 127) / 128, L.nlev);
    mg::k_resid9<T, B><<<g2, 128, 0, s>>>(L, V::t2(d), x, b, V::scratch(d, 0));
    mg::k_restrict_sum<T, O><<<dim3((dc.ncol + 127) / 128, L.nlev), 128, 0, s>>>(d.n, d.ncol, L.nlev, V::scratch(d, 0),
                                                                               V::w(d), bc, dc.ncol);
    CK(cudaGetLastError());
    return MG_OK;
}

// Algorithm 1 for the 9-cell stencil: the same steps as mgv, each a plain kernel (the
// right-hand side converted on entry and the result on exit in the FP32 variant)
template <typename T, typename B, typename O>
mg_status mgv9(mg_handle* h, const Cycle& cy, int l, const B* b, O* out, cudaStream_t s) {
    typedef View<T, T> V;
    DevLevel& d = h->lv[l];
    const size_t n = cells(h, l);
    const bool coarsest = (l == cy.L - 1);
    const double om = cy.omega;
    const T* bT = (const T*)(const void*)b;
    if (!std::is_same<B, T>::value) {
        TRY(launch_convert(h, l, n, b, V::b(d), s));
        bT = V::b(d);
    }
    T* ws[2] = {V::x(d, 0), V::x(d, 1)};
    T* cur = nullptr;
    auto other = [&]() { return cur == ws[0] ? ws[1] : ws[0]; };
    const int npre = coarsest ? cy.n_coarse : cy.n_pre;
    for (int i = 0; i < npre; ++i) {
        T* dst = other();
        TRY((sweep9<T, T, T>(h, l, cur, bT, dst, om, s)));
        cur = dst;
    }
    if (!coarsest) {
        DevLevel& dc = h->lv[l + 1];
        TRY((restrict9<T, T, T>(h, l, cur, bT, V::b(dc), s)));
        T* xc = V::r(dc);
        TRY((mgv9<T, T, T>(h, cy, l + 1, V::b(dc), xc, s)));
        T* dst = other();
        if (cur) TRY((launch_prolong<T, false, T, T>(h, l, d.n, d.ncol, dc.ncol, h->nlev, cur, xc, dst, s)));
        else TRY((launch_prolong<T, true, T, T>(h, l, d.n, d.ncol, dc.ncol, h->nlev, cur, xc, dst, s)));
        cur = dst;
        for (int i = 0; i < cy.n_post; ++i) {
            T* dst2 = other();
            TRY((sweep9<T, T, T>(h, l, cur, bT, dst2, om, s)));
            cur = dst2;
        }
    }
    if (!cur) {
        CK(cudaMemsetAsync(out, 0, n * sizeof(O), s));
        return MG_OK;
    }
    return launch_convert(h, l, n, (const T*)cur, out, s);
}

mg_status run_cycle(mg_handle* h, const Cycle& cy, const double* b, double* x, cudaStream_t s) {
    if (h->nine) {
        switch (h->prm.vcycle_precision) {
            case MG_FP64: return mgv9<double, double, double>(h, cy, 0, b, x, s);
            case MG_FP32: return mgv9<float, double, double>(h, cy, 0, b, x, s);   // (MG_FP32_P64: not built)
            default: return MG_ERR_UNSUPPORTED;
        }
    }
    switch (h->prm.vcycle_precision) {
        case MG_FP64: return mgv<double, double, double, double>(h, cy, 0, b, x, s);
        case MG_FP32:
        case MG_FP32_P64: return mgv<float, float, double, double>(h, cy, 0, b, x, s);
        case MG_FP32_BF16COEF: return mgv<float, bf16, double, double>(h, cy, 0, b, x, s);
        default: return MG_ERR_ARG;
    }
}

mg_status run_vcycle(mg_handle* h, const double* b, double* x, cudaStream_t s) {
    return run_cycle(h, vcycle_of(h), b, x, s);
}

// P_H^(Jac)(omega, n) of Sec. 4.1: n block-Jacobi sweeps from zero on the finest level, in the
// handle's V-cycle precision (a one-level cycle)
mg_status run_jacobi(mg_handle* h, double omega, int sweeps, const double* b, double* x, cudaStream_t s) {
    return run_cycle(h, Cycle{1, omega, 0, 0, sweeps}, b, x, s);
}

// BiCGStab(H, P, tol) on the finest level (Sec. 4.1 solver list; Table 1 "Krylov" rows) from
// x = 0: the vector updates and inner products run in the kernels above with device scalars;
// the host reads them once per iteration to test convergence.  *iters counts a half step as 0.5.
template <typename Pre>
mg_status bicgstab(mg_handle* h, const double* b, double* x, double tol, int maxit, Pre& P, cudaStream_t s,
                   double* iters) {
    const size_t n = cells(h, 0);
    double *rh = h->bv[0], *r = h->bv[1], *p = h->bv[2], *v = h->bv[3], *sv = h->bv[4], *t = h->bv[5],
           *ph = h->bv[6], *sh = h->bv[7];
    if (!rh) return MG_ERR_UNSUPPORTED;
    const Lvl<double, double> L = View<double, double>::lvl(h, 0);
    const dim3 ag((L.ncol + 127) / 128, L.nlev);
    const int G = h->red_grid, B = mg::RED_THREADS;
    unsigned int* tk = h->tickets + TK_BICG;
    auto apply = [&](const double* in, double* out) -> mg_status {
        if (h->nine) return launch_apply9(h, 0, in, out, s);
        Prof pr(h, MG_K_APPLY, 0, 8.0 * n * 9, s);
        mg::k_apply_a6<<<ag, 128, 0, s>>>(L, h->a6, in, out);
        CK(cudaGetLastError());
        return MG_OK;
    };
    *iters = 0.0;
    mg::k_bicg_start<<<G, B, 0, s>>>(n, b, r, rh, x, tol, h->partials, tk, h->bs);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->host_bs, h->bs, sizeof(mg::BicgScal), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!std::isfinite(h->host_bs->bb)) return MG_ERR_BREAKDOWN;
    if (h->host_bs->bb == 0.0) return MG_OK;
    for (int i = 0; i < maxit; ++i) {
        mg::k_bicg_dir<<<G, B, 0, s>>>(n, r, v, p, i == 0, h->bs);
        CK(cudaGetLastError());
        TRY(P(p, ph));
        TRY(apply(ph, v));
        mg::k_bicg_alpha<<<G, B, 0, s>>>(n, rh, v, h->partials, tk, h->bs);
        mg::k_bicg_s<<<G, B, 0, s>>>(n, r, v, sv, h->partials, tk, h->bs);
        CK(cudaGetLastError());
        TRY(P(sv, sh));
        TRY(apply(sh, t));
        mg::k_bicg_omega<<<G, B, 0, s>>>(n, t, sv, h->partials, tk, h->bs);
        mg::k_bicg_xr<<<G, B, 0, s>>>(n, x, r, ph, sh, sv, t, rh, h->partials, tk, h->bs);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h->host_bs, h->bs, sizeof(mg::BicgScal), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const mg::BicgScal& S = *h->host_bs;
        if (!std::isfinite(S.alpha) || !std::isfinite(S.ss)) return MG_ERR_BREAKDOWN;
        if (S.half) {
            *iters = i + 0.5;
            return MG_OK;
        }
        if (!std::isfinite(S.omega) || !std::isfinite(S.rr) || !std::isfinite(S.rho)) return MG_ERR_BREAKDOWN;
        *iters = i + 1.0;
        if (S.rr <= S.tol2bb) return MG_OK;
        if (S.omega == 0.0 || S.rho == 0.0) return MG_ERR_BREAKDOWN;
    }
    return MG_ERR_NOT_CONVERGED;
}

// x ~ H^-1 b by the handle's pressure solver: one V-cycle (MG(L)), line relaxation, or
// BiCGStab to eps_H preconditioned by one of the two (Table 1); *iters as for bicgstab
mg_status run_pressure_solver(mg_handle* h, const double* b, double* x, cudaStream_t s, double* iters) {
    const mg_pressure_solver& ps = h->ps;
    *iters = 0.0;
    mg_status st = MG_OK;
    switch (ps.kind) {
        case MG_PS_MG: st = run_vcycle(h, b, x, s); break;
        case MG_PS_JACOBI: st = run_jacobi(h, ps.omega, ps.sweeps, b, x, s); break;
        case MG_PS_BICGSTAB_JACOBI: {
            auto P = [&](const double* in, double* out) { return run_jacobi(h, ps.omega, ps.sweeps, in, out, s); };
            st = bicgstab(h, b, x, ps.eps, ps.max_iter, P, s, iters);
            break;
        }
        case MG_PS_BICGSTAB_MG: {
            auto P = [&](const double* in, double* out) { return run_vcycle(h, in, out, s); };
            st = bicgstab(h, b, x, ps.eps, ps.max_iter, P, s, iters);
            break;
        }
        default: return MG_ERR_ARG;
    }
    if (ps.kind == MG_PS_BICGSTAB_JACOBI || ps.kind == MG_PS_BICGSTAB_MG) {
        h->ps_solves += 1;
        h->ps_iters += *iters;
    }
    return st;
}

// the pressure solver synchronises with the host (BiCGStab): the mixed GCR then launches its
// iterations directly instead of capturing them into graphs
inline bool ps_syncs(const mg_handle* h) {
    return h->ps.kind == MG_PS_BICGSTAB_JACOBI || h->ps.kind == MG_PS_BICGSTAB_MG;
}

// ---- GCR (Sec. 4.1; textbook generalised conjugate residual, right preconditioned) ----
// Per iteration j of a restart cycle: z_j = P r (raw), w_j = A z_j with the inner products
// <w_j, w_i>, <r, w_i>, <w_j, w_j>, <r, w_j> fused into the same pass (coefficients by
// classical Gram-Schmidt), then one pass orthogonalises w_j in place and updates r with
// <r, r>.  x is formed from the raw z_i once per cycle (or at the end).
// Run-time direction count j -> kernel instantiated for exactly j directions.
template <template <int> class K, typename... A>
mg_status dispatch_j(int j, A&&... a) {
    switch (j) {
#define MG_J(n) \
    case n: return K<n>::run(std::forward<A>(a)...);
        MG_J(0) MG_J(1) MG_J(2) MG_J(3) MG_J(4) MG_J(5) MG_J(6) MG_J(7)
        MG_J(8) MG_J(9) MG_J(10) MG_J(11) MG_J(12) MG_J(13) MG_J(14) MG_J(15)
#undef MG_J
        default: return MG_ERR_ARG;
    }
}

// column-chunk of the fused apply: long enough to amortise the per-thread reduction
constexpr int GCR_APPLY_KCHUNK = 24;

template <int J>
struct RunSums {
    static mg_status run(mg_handle* h, size_t n, const double* w, cudaStream_t s) {
        Prof pr(h, MG_K_GCR_DOTS, 0, 8.0 * n * (J + 2), s);   // w, r, w_i
        mg::k_gcr_sums<J><<<h->red_grid, mg::RED_THREADS, 0, s>>>(n, w, h->W, h->glen, h->r, h->partials,
                                                                   h->tickets + TK_SUMS, h->gs);
        CK(cudaGetLastError());
        return MG_OK;
    }
};

template <int J>
struct RunApplyGcr {
    static mg_status run(mg_handle* h, const double* z, double* w, cudaStream_t s) {
        const Lvl<double, double> L = View<double, double>::lvl(h, 0);
        const double nc = (double)L.nlev * L.ncol;
        // z, the couplings (6, and the diagonal in diagonal form), w, r, w_i
        Prof pr(h, MG_K_APPLY, 0, nc * 8.0 * (1 + 6 + MG_APPLY_DIAG + 1 + 1 + J), s, J);
        const int kc = GCR_APPLY_KCHUNK;
        dim3 grid((L.ncol + mg::RED_THREADS - 1) / mg::RED_THREADS, (L.nlev + kc - 1) / kc);
        mg::k_apply_gcr<J><<<grid, mg::RED_THREADS, 0, s>>>(L, h->a6, z, w, h->W, h->glen, h->r, kc, h->partials,
                                                            h->tickets + TK_SUMS, h->gs);
        CK(cudaGetLastError());
        return MG_OK;
    }
};

template <int J>
struct RunOrth {
    static mg_status run(mg_handle* h, size_t n, cudaStream_t s) {
        Prof pr(h, MG_K_GCR_ORTH, 0, 8.0 * n * (J > 0 ? J + 4 : 3), s);
        mg::k_gcr_orth_update<J><<<h->red_grid, mg::RED_THREADS, 0, s>>>(n, h->W, h->glen, h->r, h->partials,
                                                                         h->tickets + TK_ORTH, h->gs);
        CK(cudaGetLastError());
        return MG_OK;
    }
};

template <int J>
struct RunXupd {
    static mg_status run(mg_handle* h, size_t n, double* x, cudaStream_t s) {
        Prof pr(h, MG_K_GCR_UPDATE, 0, 8.0 * n * (J + 3), s);
        mg::k_gcr_xupdate<J><<<h->red_grid, mg::RED_THREADS, 0, s>>>(n, x, h->Z, h->glen, h->gs);
        CK(cudaGetLastError());
        return MG_OK;
    }
};

mg_status gcr_sums(mg_handle* h, size_t n, const double* w, int j, cudaStream_t s) {
    return dispatch_j<RunSums>(j, h, n, w, s);
}

mg_status apply_gcr(mg_handle* h, const double* z, double* w, int j, cudaStream_t s) {
    if (h->nine) {
        TRY(launch_apply9(h, 0, z, w, s));
        return gcr_sums(h, cells(h, 0), w, j, s);
    }
    return dispatch_j<RunApplyGcr>(j, h, z, w, s);
}

// Capture the launches of `body` into *out (left null, and graphs switched off for the
// handle, if the capture or the instantiation fails; the caller then launches directly).
template <typename Body>
void capture_graph(mg_handle* h, Body& body, cudaGraphExec_t* out) {
    *out = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const mg_status st = body(h->cap);
        const cudaError_t e = cudaStreamEndCapture(h->cap, &g);
        if (st == MG_OK && e == cudaSuccess && g && cudaGraphInstantiate(out, g, 0) != cudaSuccess) *out = nullptr;
        if (g) cudaGraphDestroy(g);
    }
    if (!*out) {
        h->graphs_off = true;
        cudaGetLastError();
    }
}

// One GCR solve as resumable steps, so that several solves (an ensemble of handles) can
// interleave their iterations on their own streams: start (enqueue r = b, x = 0, <b, b>),
// started (after a synchronisation: read <b, b>), launch (enqueue one iteration, ending with
// the read-back of <r, r>), landed (after a synchronisation: read <r, r>, decide, enqueue the
// solution update when the cycle ends or the solve stops), end (enqueue the closing event).
struct GcrRun {
    int sys = 0;          // 0 pressure, 1 mixed, 2 mixed adjoint: selects the handle's cached graphs
    size_t n = 0;
    double* x = nullptr;
    double tol = 0.0;
    double bb = 0.0, rel = 0.0;
    int it = 0;
    mg_status st = MG_OK;
    bool active = false;  // iterations left to launch
};

mg_status gcr_start(mg_handle* h, GcrRun& g, const double* b, cudaStream_t s) {
    CK(cudaEventRecord(h->ev0, s));
    CK(cudaMemcpyAsync(h->r, b, g.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(g.x, 0, g.n * sizeof(double), s));
    {
        Prof pr(h, MG_K_DOT, 0, 8.0 * g.n, s);
        mg::k_dot<<<h->red_grid, mg::RED_THREADS, 0, s>>>(g.n, b, b, h->partials, h->tickets + TK_DOT, &h->gs->bb);
        CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(h->host_sc, &h->gs->bb, sizeof(double), cudaMemcpyDeviceToHost, s));
    return MG_OK;
}

void gcr_started(mg_handle* h, GcrRun& g) {
    g.bb = h->host_sc[0];
    g.it = 0;
    g.rel = 0.0;
    g.active = false;
    g.st = MG_OK;
    if (!std::isfinite(g.bb)) {
        g.st = MG_ERR_BREAKDOWN;
    } else if (g.bb > 0.0) {
        g.rel = 1.0;
        g.st = MG_ERR_NOT_CONVERGED;
        g.active = h->prm.max_iter > 0;
    }
}

template <typename ApplyAS, typename ApplyP>
mg_status gcr_launch(mg_handle* h, GcrRun& g, cudaStream_t s, ApplyAS& applyAS, ApplyP& applyP) {
    const int j = g.it % h->prm.gcr_restart;
    double* z = h->Z + (size_t)j * h->glen;
    double* w = h->W + (size_t)j * h->glen;
    const size_t n = g.n;
    // every buffer of the iteration belongs to the handle, so its launches form a fixed
    // sequence per slot j
    auto body = [&](cudaStream_t q) -> mg_status {
        TRY(applyP(h->r, z, q));
        TRY(applyAS(z, w, j, q));
        TRY(dispatch_j<RunOrth>(j, h, n, q));
        CK(cudaMemcpyAsync(h->host_sc, &h->gs->rr, sizeof(double), cudaMemcpyDeviceToHost, q));
        return MG_OK;
    };
    cudaGraphExec_t& ge = h->gexec[g.sys][j];
    const bool direct = h->prof || (g.sys != 0 && ps_syncs(h));
    if (!ge && !direct && !h->graphs_off) capture_graph(h, body, &ge);
    if (ge && !direct) CK(cudaGraphLaunch(ge, s));
    else TRY(body(s));
    return MG_OK;
}

mg_status gcr_landed(mg_handle* h, GcrRun& g, cudaStream_t s) {
    const int j = g.it % h->prm.gcr_restart;
    ++g.it;
    const double rr = h->host_sc[0];
    if (!std::isfinite(rr)) {
        g.st = MG_ERR_BREAKDOWN;
        g.active = false;
        return MG_OK;
    }
    g.rel = std::sqrt(rr / g.bb);
    const bool done = g.rel <= g.tol;
    if (j == h->prm.gcr_restart - 1 || done || g.it == h->prm.max_iter)
        TRY(dispatch_j<RunXupd>(j, h, g.n, g.x, s));
    if (done) g.st = MG_OK;
    g.active = !done && g.it < h->prm.max_iter;
    return MG_OK;
}

void gcr_info(mg_handle* h, const GcrRun& g, mg_solve_info* info) {
    if (!info) return;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    info->iters = g.it;
    info->rel_res = g.rel;
    info->ms = ms;
}

template <typename ApplyAS, typename ApplyP>
mg_status gcr(mg_handle* h, int sys, size_t n, const double* b, double* x, double tol, mg_solve_info* info,
              cudaStream_t s, ApplyAS applyAS, ApplyP applyP) {
    GcrRun g;
    g.sys = sys;
    g.n = n;
    g.x = x;
    g.tol = tol;
    TRY(gcr_start(h, g, b, s));
    CK(cudaStreamSynchronize(s));
    gcr_started(h, g);
    while (g.active) {
        NvtxRange it_("gcr iteration");
        TRY(gcr_launch(h, g, s, applyAS, applyP));
        CK(cudaStreamSynchronize(s));
        TRY(gcr_landed(h, g, s));
    }
    CK(cudaEventRecord(h->ev1, s));
    CK(cudaEventSynchronize(h->ev1));
    gcr_info(h, g, info);
    return g.st;
}

// ---- mixed operator and Schur-complement preconditioner ----
mg_status mixed_apply_impl(mg_handle* h, const double* u, const double* p, double* yu, double* yp, cudaStream_t s) {
    const mg::MixedDev& M = h->md;
    const size_t nh = (size_t)M.nlev * M.nfh;
    const int bd = 128;
    Prof pr(h, MG_K_MIXED, 0, 8.0 * (2.0 * h->nu + 3.0 * cells(h, 0)), s);
    mg::k_mx_faces_h<0><<<dim3((M.nfh + bd - 1) / bd, M.nlev), bd, 0, s>>>(M, u, p, yu);
    mg::k_mx_faces_v<0><<<dim3((M.ncol + bd - 1) / bd, M.nlev + 1), bd, 0, s>>>(M, u + nh, p, yu + nh);
    mg::k_mx_cells<0><<<dim3((M.ncol + bd - 1) / bd, M.nlev), bd, 0, s>>>(M, u, u + nh, p, yp);
    CK(cudaGetLastError());
    return MG_OK;
}

// A-hat [u; p]: the mixed operator with its velocity mass replaced by W^-1 M-bar^T W
mg_status mixed_apply_hat_impl(mg_handle* h, const double* u, const double* p, double* yu, double* yp,
                               cudaStream_t s) {
    const mg::MixedDev& M = h->md;
    const size_t nh = (size_t)M.nlev * M.nfh;
    const int bd = 128;
    Prof pr(h, MG_K_MIXED, 0, 8.0 * (3.0 * h->nu + 3.0 * cells(h, 0)), s, 2);
    mg::k_mx_faces_h<2><<<dim3((M.nfh + bd - 1) / bd, M.nlev), bd, 0, s>>>(M, u, p, yu);
    mg::k_mx_faces_v<2><<<dim3((M.ncol + bd - 1) / bd, M.nlev + 1), bd, 0, s>>>(M, u + nh, p, yu + nh);
    mg::k_mx_cells<0><<<dim3((M.ncol + bd - 1) / bd, M.nlev), bd, 0, s>>>(M, u, u + nh, p, yp);
    CK(cudaGetLastError());
    return MG_OK;
}

template <bool MULT>
mg_status mixed_adj_scale(mg_handle* h, const double* in_u, const double* in_p, double* out_u, double* out_p,
                          cudaStream_t s) {
    Prof pr(h, MG_K_DOT, 0, 16.0 * ((double)h->nu + (double)cells(h, 0)), s, MULT ? 1 : 0);
    mg::k_mx_adj_scale<MULT><<<4 * h->nsm, 256, 0, s>>>(h->md, (size_t)h->nu, h->area0, h->dz, in_u, in_p, out_u,
                                                          out_p);
    CK(cudaGetLastError());
    return MG_OK;
}

mg_status schur_impl(mg_handle* h, const double* ru, const double* rp, double* u, double* p, cudaStream_t s) {
    const mg::MixedDev& M = h->md;
    const size_t nh = (size_t)M.nlev * M.nfh;
    const int bd = 128;
    // Step 1: B = r_p - D M-ring^{-1} r_u
    mg::k_mx_cells<1><<<dim3((M.ncol + bd - 1) / bd, M.nlev), bd, 0, s>>>(M, ru, ru + nh, rp, h->schurB);
    CK(cudaGetLastError());
    // Step 2: H Pi' = B by the pressure solver K_H(A_H, P_H, eps_H) (one V-cycle by default);
    // an inexact inner solve (BiCGStab at its iteration limit) is still a usable preconditioner
    double it = 0.0;
    const mg_status st = run_pressure_solver(h, h->schurB, p, s, &it);
    if (st != MG_OK && st != MG_ERR_NOT_CONVERGED) return st;
    // Step 3: u' = M-ring^{-1} (r_u - G Pi')
    mg::k_mx_faces_h<1><<<dim3((M.nfh + bd - 1) / bd, M.nlev), bd, 0, s>>>(M, ru, p, u);
    mg::k_mx_faces_v<1><<<dim3((M.ncol + bd - 1) / bd, M.nlev + 1), bd, 0, s>>>(M, ru + nh, p, u + nh);
    CK(cudaGetLastError());
    return MG_OK;
}

// Replaces the finest-level operator by the caller's couplings a[s][k][c] (DEVICE, 6 N): the
// FP64 operator of the GCR apply takes them as they are, the V-cycle's finest level their face
// form in its precision.  A first pass only checks them (flux symmetry, sign, no flux through
// surface and lid); the operator is changed only if every check passes.
mg_status set_coefficients_impl(mg_handle* h, const double* a, cudaStream_t s) {
    const int ncol = h->lv[0].ncol, nlev = h->nlev, nf = 2 * ncol;
    const DevLevel& d = h->lv[0];
    const mg::CoefTargets t{d.Th64, d.Th32, d.Th16, d.Tv64, d.Tv32, d.Tv16};
    CK(cudaMemsetAsync(h->flag, 0, sizeof(unsigned int), s));
    for (int pass = 0; pass < 2; ++pass) {
        const bool write = pass == 1;
        mg::k_coef_faces<<<dim3((nf + 127) / 128, nlev), 128, 0, s>>>(ncol, nlev, h->faceL0, h->faceR0, h->faceSide0,
                                                                       h->nbrSide0, h->area0, a, write, t, h->flag);
        mg::k_coef_vertical<<<dim3((ncol + 127) / 128, nlev + 1), 128, 0, s>>>(ncol, nlev, h->dz, a, write, t,
                                                                                h->flag);
        CK(cudaGetLastError());
        if (!write) {
            unsigned int bad = 0;
            CK(cudaMemcpyAsync(&bad, h->flag, sizeof bad, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (bad) return MG_ERR_ARG;
        }
    }
    mg::k_coef_cells<<<4 * h->nsm, 256, 0, s>>>(cells(h, 0), a, h->a6);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return MG_OK;
}

mg_status check_level(const mg_handle* h, int level) {
    if (!h || level < 0 || level >= h->L) return MG_ERR_ARG;
    return MG_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Horizontal-face velocity mass M_h = M2 + tau_u dt M_C of the mixed system (level-
// independent): the self weight, up to 6 couplings per face (the opposite face in each of
// its two cells, then the two perpendicular faces in each) and the lumped diagonal.
struct HMass {
    int ncf = 0;                  // couplings per face (0 or 6)
    double ms = 1.0;              // self weight (2/3 consistent, 1 lumped)
    std::vector<int32_t> cf;      // [6][nfh] coupled face
    std::vector<double> wf;       // [6][nfh] its weight
    std::vector<double> mlump;    // [nfh] row sums in the cells' own axes
};

void horizontal_mass(const mg::HGeom& G, bool consistent, double f0, HMass& hm) {
    const int ncol = G.ncol, nfh = 2 * ncol;
    const double outward[4] = {1.0, -1.0, 1.0, -1.0};   // E, W, N, S along +xi, -xi, +eta, -eta
    hm.ms = consistent ? 2.0 / 3.0 : 1.0;
    hm.ncf = (consistent || f0 != 0.0) ? 6 : 0;
    hm.mlump.assign(nfh, 0.0);
    hm.cf.assign((size_t)hm.ncf * nfh, 0);
    hm.wf.assign((size_t)hm.ncf * nfh, 0.0);
    // sign of the normal of face (side s of column c) along the cell's axis
    auto tau = [&](int c, int s) {
        const int f = G.face_of[s * ncol + c];
        return outward[s] * (G.faceL[f] == c ? 1.0 : -1.0);
    };
    for (int f = 0; f < nfh; ++f) {
        const int cells[2] = {G.faceL[f], G.faceR[f]};
        const int sides[2] = {G.faceSide[f], G.nbr_side[G.faceSide[f] * ncol + G.faceL[f]]};
        double lump = 0.0;
        for (int e = 0; e < 2; ++e) {
            const int c = cells[e], a = sides[e];
            const bool xi = a < 2;
            const double Fc = f0 * G.sinlat[c], ta = tau(c, a);
            // element row sum: 1/3 + 1/6 (or the lumped 1/2) and -+ 2 F_c / 4
            lump += 0.5 + (xi ? -0.5 : 0.5) * Fc;
            if (hm.ncf == 0) continue;
            const int b = a ^ 1;   // opposite side
            hm.cf[(size_t)e * nfh + f] = G.face_of[b * ncol + c];
            hm.wf[(size_t)e * nfh + f] = consistent ? ta * tau(c, b) / 6.0 : 0.0;
            const int p0 = xi ? 2 : 0;   // perpendicular sides
            for (int t = 0; t < 2; ++t) {
                const int bp = p0 + t;
                const size_t slot = (size_t)(2 + 2 * e + t) * nfh + f;
                hm.cf[slot] = G.face_of[bp * ncol + c];
                hm.wf[slot] = ta * tau(c, bp) * Fc * (xi ? -0.25 : 0.25);
            }
        }
        hm.mlump[f] = lump;
    }
}

mg_status setup_impl(mg_handle* h, const mg_mesh* mesh, const mg_params* prm, const double* g,
                     const mg_mixed* mixed, double gamma2 = 0.0) {
    const int L = prm->levels, n = mesh->n, nlev = mesh->nlev;
    h->L = L;
    h->n = n;
    h->nlev = nlev;
    h->prm = *prm;
    CK(cudaGetDevice(&h->device));
    CK(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device));
    h->red_grid = 8 * h->nsm;
    // host hierarchy
    std::vector<mg::HGeom> hg(L);
    for (int l = 0; l < L; ++l) {
        const std::string err = mg::build_hgeom(n >> l, mesh->radius, hg[l]);
        if (!err.empty()) return MG_ERR_ARG;
    }
    mg::VGeom vg;
    if (!mg::build_vgeom(mesh->z_interfaces, nlev, vg).empty()) return MG_ERR_ARG;
    const int ncol0 = hg[0].ncol;
    const size_t N0 = (size_t)nlev * ncol0, NV0 = (size_t)(nlev + 1) * ncol0;
    std::vector<mg::LevelCoef> co(L);
    co[0].g.assign(g, g + N0);
    for (size_t i = 0; i < N0; ++i)
        if (!(g[i] > 0.0) || !std::isfinite(g[i])) return MG_ERR_ARG;
    co[0].mu.assign(NV0, 1.0);
    std::vector<double> w_up, w_dn;
    HMass hm;
    double mv = 1.0;
    if (mixed) {
        // vertical faces: consistent mass 2/3 on the face and 1/6 to the interior faces
        // above and below, plus eps B_w; lumped to the row sums
        const double off = mixed->consistent ? 1.0 / 6.0 : 0.0;
        mv = mixed->consistent ? 2.0 / 3.0 : 1.0;
        w_up.assign(NV0, 0.0);
        w_dn.assign(NV0, 0.0);
        for (int kf = 1; kf < nlev; ++kf) {
            for (int c = 0; c < ncol0; ++c) {
                const size_t o = (size_t)kf * ncol0 + c;
                if (kf + 1 <= nlev - 1) w_up[o] = mixed->eps * mixed->beta_up[o] + off;
                if (kf - 1 >= 1) w_dn[o] = mixed->eps * mixed->beta_dn[o] + off;
                co[0].mu[o] = 1.0 / (mv + w_up[o] + w_dn[o]);   // 1 / row sum
            }
        }
        horizontal_mass(hg[0], mixed->consistent != 0, mixed->coriolis_f0, hm);
        co[0].muh.resize(hm.mlump.size());
        for (size_t f = 0; f < hm.mlump.size(); ++f) co[0].muh[f] = 1.0 / hm.mlump[f];
    }
    for (int l = 1; l < L; ++l) {
        co[l].g.resize((size_t)nlev * hg[l].ncol);
        co[l].mu.resize((size_t)(nlev + 1) * hg[l].ncol);
        mg::restrict_mean(hg[l - 1], hg[l], nlev, co[l - 1].g.data(), co[l].g.data());
        mg::restrict_mean(hg[l - 1], hg[l], nlev + 1, co[l - 1].mu.data(), co[l].mu.data());
        if (!co[l - 1].muh.empty()) {
            co[l].muh.resize(2 * (size_t)hg[l].ncol);
            mg::restrict_face_mean(hg[l - 1], hg[l], co[l - 1].muh.data(), co[l].muh.data());
        }
    }
    for (int l = 0; l < L; ++l) mg::level_coefficients(hg[l], vg, mesh->cs_dt, co[l]);
    // upload
    std::vector<double> rdz(nlev);
    for (int k = 0; k < nlev; ++k) rdz[k] = 1.0 / vg.dz[k];
    TRY(upload(h, &h->rdz64, rdz));
    TRY(upload(h, &h->dz, vg.dz));
    TRY(upload(h, &h->area0, hg[0].area));
    TRY(upload(h, &h->rdz32, rdz));
    TRY(upload(h, &h->faceL0, hg[0].faceL));
    TRY(upload(h, &h->faceR0, hg[0].faceR));
    TRY(upload(h, &h->faceSide0, hg[0].faceSide));
    TRY(upload(h, &h->nbrSide0, hg[0].nbr_side));
    TRY(dalloc(h, &h->flag, 1));
    // MG_FP32_P64 stores and computes as MG_FP32; only the finest level's elimination differs
    const int prec = prm->vcycle_precision == MG_FP32_P64 ? MG_FP32 : prm->vcycle_precision;
    h->pivot64 = prm->vcycle_precision == MG_FP32_P64;
    h->lv.resize(L);
    for (int l = 0; l < L; ++l) {
        DevLevel& d = h->lv[l];
        const mg::HGeom& G = hg[l];
        d.n = G.n;
        d.ncol = G.ncol;
        std::vector<double> rA(G.ncol);
        for (int c = 0; c < G.ncol; ++c) rA[c] = 1.0 / G.area[c];
        TRY(upload(h, &d.nbr, G.nbr));
        TRY(upload(h, &d.fof, G.face_of));
        TRY(upload(h, &d.rA64, rA));
        TRY(upload(h, &d.Th64, co[l].Th));
        TRY(upload(h, &d.Tv64, co[l].Tv));
        const size_t Nl = (size_t)nlev * G.ncol;
        TRY(dalloc(h, &d.x64[0], Nl));
        TRY(dalloc(h, &d.x64[1], Nl));
        TRY(dalloc(h, &d.b64, Nl));
        TRY(dalloc(h, &d.r64, Nl));
        if (prec != MG_FP64) {
            TRY(upload(h, &d.rA32, rA));
            if (prec == MG_FP32) {
                TRY(upload(h, &d.Th32, co[l].Th));
                TRY(upload(h, &d.Tv32, co[l].Tv));
            } else {
                TRY(upload(h, &d.Th16, co[l].Th));
                TRY(upload(h, &d.Tv16, co[l].Tv));
            }
            TRY(dalloc(h, &d.x32[0], Nl));
            TRY(dalloc(h, &d.x32[1], Nl));
            TRY(dalloc(h, &d.b32, Nl));
            TRY(dalloc(h, &d.r32, Nl));
        }
        if (gamma2 > 0.0) {
            // 9-cell stencil: flux between cells k and k + 2 of every column,
            // gamma2 (c_s dt)^2 (g_k + g_k+2) / 2 / (z_c[k+2] - z_c[k])
            h->nine = true;
            std::vector<double> t2(Nl, 0.0);
            const double c2 = mesh->cs_dt * mesh->cs_dt;
            const double* z = mesh->z_interfaces;
            for (int k = 0; k + 2 < nlev; ++k) {
                const double dzc2 = 0.5 * (z[k + 3] + z[k + 2]) - 0.5 * (z[k + 1] + z[k]);
                for (int c = 0; c < G.ncol; ++c)
                    t2[(size_t)k * G.ncol + c] =
                        gamma2 * c2 * 0.5 * (co[l].g[(size_t)k * G.ncol + c] + co[l].g[(size_t)(k + 2) * G.ncol + c]) /
                        dzc2;
            }
            TRY(upload(h, &d.T2_64, t2));
            for (double*& p : d.s64) TRY(dalloc(h, &p, Nl));
            if (prec == MG_FP32) {
                TRY(upload(h, &d.T2_32, t2));
                for (float*& p : d.s32) TRY(dalloc(h, &p, Nl));
            }
        }
        if (l + 1 < L) {
            const mg::HGeom& Gc = hg[l + 1];
            std::vector<double> w(4 * (size_t)Gc.ncol);
            for (int C = 0; C < Gc.ncol; ++C)
                for (int q = 0; q < 4; ++q) w[(size_t)q * Gc.ncol + C] = G.area[mg::child_col(G.n, C, q)] / Gc.area[C];
            TRY(upload(h, &d.w64, w));
            if (prec != MG_FP64) TRY(upload(h, &d.w32, w));
        }
    }
    {
        // finest level: a_side = Th[k][face] / area, a_up = Tv[k+1] / dz, a_dn = Tv[k] / dz,
        // and the diagonal 1 + sum of the six
        const mg::HGeom& G = hg[0];
        const size_t N = (size_t)nlev * ncol0;
        std::vector<double> a6(7 * N);
        for (int k = 0; k < nlev; ++k)
            for (int c = 0; c < ncol0; ++c) {
                const size_t e = (size_t)k * ncol0 + c;
                const double rA = 1.0 / G.area[c];
                for (int sd = 0; sd < 4; ++sd)
                    a6[sd * N + e] = co[0].Th[(size_t)k * 2 * ncol0 + G.face_of[sd * ncol0 + c]] * rA;
                a6[4 * N + e] = co[0].Tv[(size_t)(k + 1) * ncol0 + c] * rdz[k];
                a6[5 * N + e] = co[0].Tv[(size_t)k * ncol0 + c] * rdz[k];
                double d = 1.0;
                for (int f = 0; f < 6; ++f) d += a6[f * N + e];
                a6[6 * N + e] = d;
            }
        TRY(upload(h, &h->a6, a6));
    }
    // mixed system arrays (finest level)
    h->mixed = mixed != nullptr;
    if (h->mixed) {
        const mg::HGeom& G = hg[0];
        const int nfh = 2 * ncol0;
        // gradient and divergence each carry one factor c_s dt; their product is the
        // Helmholtz coupling (c_s dt)^2 g_f A_f / (V_i d_f)
        const double c = mesh->cs_dt;
        std::vector<double> kd_h((size_t)nlev * nfh), kd_v(NV0, 0.0), sdiv(4 * (size_t)ncol0), divv(nlev);
        for (int k = 0; k < nlev; ++k) divv[k] = c / vg.dz[k];
        for (int f = 0; f < nfh; ++f) {
            const int Lc = G.faceL[f], Rc = G.faceR[f], sd = G.faceSide[f];
            const double dist = G.cdist[sd * ncol0 + Lc];
            for (int k = 0; k < nlev; ++k)
                kd_h[(size_t)k * nfh + f] = c * 0.5 * (g[(size_t)k * ncol0 + Lc] + g[(size_t)k * ncol0 + Rc]) / dist;
        }
        for (int kf = 1; kf < nlev; ++kf)
            for (int col = 0; col < ncol0; ++col)
                kd_v[(size_t)kf * ncol0 + col] =
                    c * 0.5 * (g[(size_t)(kf - 1) * ncol0 + col] + g[(size_t)kf * ncol0 + col]) / vg.dzc[kf];
        for (int col = 0; col < ncol0; ++col)
            for (int sd = 0; sd < 4; ++sd) {
                const int f = G.face_of[sd * ncol0 + col];
                const double sgn = (G.faceL[f] == col) ? 1.0 : -1.0;
                sdiv[(size_t)sd * ncol0 + col] = sgn * c * G.edge_len[sd * ncol0 + col] / G.area[col];
            }
        // adjoint: face weights W_f = A_f d_f / g_f and the rows of M_h^T.  The surface and lid
        // faces are decoupled identity rows, so any weight keeps A^T = S J A-hat J S^-1; they
        // take area dz / g of their cell, the size of the interior weights (a weight far from
        // those would let their entries dominate the residual norm of the scaled system)
        std::vector<double> Wf((size_t)nlev * nfh + NV0, 1.0);
        for (int col = 0; col < ncol0; ++col) {
            Wf[(size_t)nlev * nfh + col] = G.area[col] * vg.dz[0] / g[col];
            Wf[(size_t)nlev * nfh + (size_t)nlev * ncol0 + col] =
                G.area[col] * vg.dz[nlev - 1] / g[(size_t)(nlev - 1) * ncol0 + col];
        }
        for (int f = 0; f < nfh; ++f) {
            const int Lc = G.faceL[f], Rc = G.faceR[f], sd = G.faceSide[f];
            const double el = G.edge_len[sd * ncol0 + Lc], dist = G.cdist[sd * ncol0 + Lc];
            for (int k = 0; k < nlev; ++k)
                Wf[(size_t)k * nfh + f] =
                    el * vg.dz[k] * dist / (0.5 * (g[(size_t)k * ncol0 + Lc] + g[(size_t)k * ncol0 + Rc]));
        }
        for (int kf = 1; kf < nlev; ++kf)
            for (int col = 0; col < ncol0; ++col)
                Wf[(size_t)nlev * nfh + (size_t)kf * ncol0 + col] =
                    G.area[col] * vg.dzc[kf] /
                    (0.5 * (g[(size_t)(kf - 1) * ncol0 + col] + g[(size_t)kf * ncol0 + col]));
        std::vector<double> wfT(hm.wf.size(), 0.0);
        for (int f = 0; f < nfh; ++f)
            for (int t = 0; t < hm.ncf; ++t) {
                const int gf = hm.cf[(size_t)t * nfh + f];
                int found = -1;
                for (int u = 0; u < hm.ncf; ++u)
                    if (hm.cf[(size_t)u * nfh + gf] == f) found = u;
                if (found < 0) return MG_ERR_ARG;   // the coupling pattern is symmetric by construction
                wfT[(size_t)t * nfh + f] = hm.wf[(size_t)found * nfh + gf];
            }
        std::vector<double> cdh(nfh), cdv(nlev + 1, 0.0);
        for (int f = 0; f < nfh; ++f) cdh[f] = c / (2.0 * G.cdist[G.faceSide[f] * ncol0 + G.faceL[f]]);
        for (int kf = 1; kf < nlev; ++kf) cdv[kf] = c / (2.0 * vg.dzc[kf]);
        int32_t *fL, *fR, *dcf = nullptr;
        double *dkd_h, *dkd_v, *dsdiv, *dwu, *dwd, *dml, *ddivv, *dwf = nullptr, *dmlh, *dwfT = nullptr, *dWf, *dcdh,
            *dcdv;
        TRY(upload(h, &fL, G.faceL));
        TRY(upload(h, &fR, G.faceR));
        TRY(upload(h, &dkd_h, kd_h));
        TRY(upload(h, &dkd_v, kd_v));
        TRY(upload(h, &dsdiv, sdiv));
        TRY(upload(h, &dwu, w_up));
        TRY(upload(h, &dwd, w_dn));
        TRY(upload(h, &dml, co[0].mu));     // 1 / lumped mass (1 on the boundary faces)
        TRY(upload(h, &ddivv, divv));
        TRY(upload(h, &dmlh, co[0].muh));
        if (hm.ncf > 0) {
            TRY(upload(h, &dcf, hm.cf));
            TRY(upload(h, &dwf, hm.wf));
            TRY(upload(h, &dwfT, wfT));
        }
        TRY(upload(h, &dWf, Wf));
        TRY(upload(h, &dcdh, cdh));
        TRY(upload(h, &dcdv, cdv));
        h->md = mg::MixedDev{ncol0, nlev, nfh, fL, fR, h->lv[0].fof, dsdiv, dkd_h, dkd_v, dwu, dwd, dml, ddivv,
                             hm.ncf, dcf, dwf, hm.ms, mv, dmlh, dwfT, dWf, dcdh, dcdv, mixed->eps};
        h->nu = (int64_t)nlev * nfh + (int64_t)NV0;
        TRY(dalloc(h, &h->schurB, N0));
        TRY(dalloc(h, &h->mb, (size_t)h->nu + N0));
        TRY(dalloc(h, &h->mx, (size_t)h->nu + N0));
    }
    // GCR workspace; the slot stride is padded off a multiple of large powers of two so
    // the directions streamed side by side do not share their low address bits
    h->glen = (N0 + (size_t)h->nu + 63) / 64 * 64 + 96;
    TRY(dalloc(h, &h->Z, (size_t)prm->gcr_restart * h->glen));
    TRY(dalloc(h, &h->W, (size_t)prm->gcr_restart * h->glen));
    TRY(dalloc(h, &h->r, h->glen));
    TRY(dalloc(h, &h->adj, N0));
    TRY(dalloc(h, &h->gs, 1));
    {
        const size_t apply_blocks = (size_t)((ncol0 + mg::RED_THREADS - 1) / mg::RED_THREADS) *
                                    ((nlev + GCR_APPLY_KCHUNK - 1) / GCR_APPLY_KCHUNK);
        const size_t blocks = apply_blocks > (size_t)h->red_grid ? apply_blocks : (size_t)h->red_grid;
        h->npartials = blocks * (2 * mg::MAXR + 2);
        TRY(dalloc(h, &h->partials, h->npartials));
    }
    TRY(dalloc(h, &h->tickets, TK_COUNT));
    CK(cudaMemset(h->tickets, 0, TK_COUNT * sizeof(unsigned int)));
    CK(cudaMemset(h->gs, 0, sizeof(mg::GcrScal)));
    if (!mem_alloc((void**)&h->host_sc, 4 * sizeof(double), MEM_PINNED)) return MG_ERR_NOMEM;
    if (!mem_alloc((void**)&h->host_bs, sizeof(mg::BicgScal), MEM_PINNED)) return MG_ERR_NOMEM;
    TRY(dalloc(h, &h->bs, 1));
    CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&h->run, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->evx, cudaEventDisableTiming));
    CK(cudaEventCreate(&h->ev0));
    CK(cudaEventCreate(&h->ev1));
    CK(cudaDeviceSynchronize());
    return MG_OK;
}

void free_handle(mg_handle* h) {
    if (!h) return;
    for (void* p : h->allocs) mem_free(p, MEM_DEVICE);
    mem_free(h->host_sc, MEM_PINNED);
    mem_free(h->host_bs, MEM_PINNED);
    for (auto& row : h->gexec)
        for (cudaGraphExec_t g : row)
            if (g) cudaGraphExecDestroy(g);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->run) cudaStreamDestroy(h->run);
    if (h->evx) cudaEventDestroy(h->evx);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
    delete h;
}

}  // namespace

// ---- an ensemble of pressure solves as one CUDA graph ----
struct mg_ensemble {
    int device = 0;
    int count = 0;
    std::vector<mg_handle*> hs;
    cudaStream_t cs = nullptr;            // capture stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    mg::EnsState* st = nullptr;           // device, one per member
    mg::EnsState* host_st = nullptr;      // pinned copy, written by the graph's last node
    unsigned long long* stamps = nullptr; // device: launch time, then every member's end [ns]
    unsigned long long* host_stamps = nullptr;
};

namespace {

void free_ensemble(mg_ensemble* e) {
    if (!e) return;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    mem_free(e->st, MEM_DEVICE);
    mem_free(e->host_st, MEM_PINNED);
    mem_free(e->stamps, MEM_DEVICE);
    mem_free(e->host_stamps, MEM_PINNED);
    if (e->cs) cudaStreamDestroy(e->cs);
    delete e;
}

// Ends the capture on e->cs and returns the nodes the next work depends on.
mg_status end_segment(mg_ensemble* e, std::vector<cudaGraphNode_t>& deps) {
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(e->cs, &cst, nullptr, nullptr, &d, nullptr, &nd));
    deps.assign(d, d + nd);
    cudaGraph_t g = nullptr;
    CK(cudaStreamEndCapture(e->cs, &g));
    return MG_OK;
}

mg_status add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle hnd,
                          cudaGraphConditionalNodeType type, cudaGraphNode_t* node, cudaGraph_t* body) {
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hnd;
    p.conditional.type = type;
    p.conditional.size = 1;
    CK(cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p));
    *body = p.conditional.phGraph_out[0];
    return MG_OK;
}

// The launches of one member: start, then WHILE { IF slot 0 {iteration}, IF {update}, ..., IF slot R-1
// {iteration}, IF {update} }, then the member's end event.
mg_status build_member(mg_ensemble* e, int i, mg_handle* h, const double* b, double* x, double tol,
                       const std::vector<cudaGraphNode_t>& root, std::vector<cudaGraphNode_t>& ends) {
    const int R = h->prm.gcr_restart;
    const size_t n = cells(h, 0);
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    mg::EnsHandles hs{};
    CK(cudaGraphConditionalHandleCreate(&hs.w, e->graph, 0, cudaGraphCondAssignDefault));
    for (int j = 0; j < R; ++j) {
        CK(cudaGraphConditionalHandleCreate(&hs.c[j], e->graph, 0, cudaGraphCondAssignDefault));
        CK(cudaGraphConditionalHandleCreate(&hs.x[j], e->graph, 0, cudaGraphCondAssignDefault));
    }
    mg::EnsState* st = e->st + i;
    // start: r = b, x = 0, <b, b>, first decision
    std::vector<cudaGraphNode_t> deps;
    CK(cudaStreamBeginCaptureToGraph(e->cs, e->graph, root.data(), nullptr, root.size(), mode));
    CK(cudaMemcpyAsync(h->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, e->cs));
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), e->cs));
    mg::k_dot<<<h->red_grid, mg::RED_THREADS, 0, e->cs>>>(n, b, b, h->partials, h->tickets + TK_DOT, &h->gs->bb);
    mg::k_ens_init<<<1, 1, 0, e->cs>>>(h->gs, st, R, h->prm.max_iter, hs);
    CK(cudaGetLastError());
    TRY(end_segment(e, deps));
    cudaGraphNode_t wnode;
    cudaGraph_t wbody;
    TRY(add_conditional(e->graph, deps, hs.w, cudaGraphCondTypeWhile, &wnode, &wbody));
    std::vector<cudaGraphNode_t> prev;
    for (int j = 0; j < R; ++j) {
        cudaGraphNode_t inode, xnode;
        cudaGraph_t ibody, xbody;
        TRY(add_conditional(wbody, prev, hs.c[j], cudaGraphCondTypeIf, &inode, &ibody));
        CK(cudaStreamBeginCaptureToGraph(e->cs, ibody, nullptr, nullptr, 0, mode));
        double* z = h->Z + (size_t)j * h->glen;
        double* w = h->W + (size_t)j * h->glen;
        TRY(run_vcycle(h, h->r, z, e->cs));
        TRY(apply_gcr(h, z, w, j, e->cs));
        TRY(dispatch_j<RunOrth>(j, h, n, e->cs));
        mg::k_ens_decide<<<1, 1, 0, e->cs>>>(h->gs, st, j, R, h->prm.max_iter, tol, hs);
        CK(cudaGetLastError());
        TRY(end_segment(e, deps));
        TRY(add_conditional(wbody, {inode}, hs.x[j], cudaGraphCondTypeIf, &xnode, &xbody));
        CK(cudaStreamBeginCaptureToGraph(e->cs, xbody, nullptr, nullptr, 0, mode));
        TRY(dispatch_j<RunXupd>(j, h, n, x, e->cs));
        TRY(end_segment(e, deps));
        prev.assign(1, xnode);
    }
    // the member's end
    CK(cudaStreamBeginCaptureToGraph(e->cs, e->graph, &wnode, nullptr, 1, mode));
    mg::k_stamp<<<1, 1, 0, e->cs>>>(e->stamps + 1 + i);
    CK(cudaGetLastError());
    TRY(end_segment(e, deps));
    ends.insert(ends.end(), deps.begin(), deps.end());
    return MG_OK;
}

mg_status build_ensemble(mg_ensemble* e, const double* const* b, double* const* x, double tol) {
    CK(cudaStreamCreateWithFlags(&e->cs, cudaStreamNonBlocking));
    if (!mem_alloc((void**)&e->st, e->count * sizeof(mg::EnsState), MEM_DEVICE) ||
        !mem_alloc((void**)&e->host_st, e->count * sizeof(mg::EnsState), MEM_PINNED) ||
        !mem_alloc((void**)&e->stamps, (e->count + 1) * sizeof(unsigned long long), MEM_DEVICE) ||
        !mem_alloc((void**)&e->host_stamps, (e->count + 1) * sizeof(unsigned long long), MEM_PINNED))
        return MG_ERR_NOMEM;
    CK(cudaGraphCreate(&e->graph, 0));
    // root: the launch time; every member starts after it
    std::vector<cudaGraphNode_t> root, deps;
    CK(cudaStreamBeginCaptureToGraph(e->cs, e->graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    mg::k_stamp<<<1, 1, 0, e->cs>>>(e->stamps);
    CK(cudaGetLastError());
    TRY(end_segment(e, root));
    std::vector<cudaGraphNode_t> ends;
    for (int i = 0; i < e->count; ++i) TRY(build_member(e, i, e->hs[i], b[i], x[i], tol, root, ends));
    // last nodes: every member's state and time stamp to the host
    CK(cudaStreamBeginCaptureToGraph(e->cs, e->graph, ends.data(), nullptr, ends.size(), cudaStreamCaptureModeThreadLocal));
    CK(cudaMemcpyAsync(e->host_st, e->st, e->count * sizeof(mg::EnsState), cudaMemcpyDeviceToHost, e->cs));
    CK(cudaMemcpyAsync(e->host_stamps, e->stamps, (e->count + 1) * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, e->cs));
    TRY(end_segment(e, deps));
    CK(cudaGraphInstantiate(&e->exec, e->graph, 0));
    return MG_OK;
}

}  // namespace

// =====================================================================================
static mg_status mg_setup_check(const mg_mesh* mesh, const mg_params* prm, const double* g, const mg_mixed* mixed);

extern "C" {

const char* mg_last_cuda_error(void) {
    return g_last_cuda == cudaSuccess ? "no CUDA error" : cudaGetErrorName(g_last_cuda);
}

int64_t mg_inject_alloc_failure(int64_t nth) {
    const long long seen = g_alloc_seen.exchange(0);
    g_fail_at.store(nth > 0 ? nth : 0);
    return seen;
}

int64_t mg_live_allocations(void) { return g_live.load(); }

const char* mg_status_string(mg_status s) {
    switch (s) {
        case MG_OK: return "ok";
        case MG_ERR_ARG: return "invalid argument";
        case MG_ERR_CUDA: return "CUDA runtime error";
        case MG_ERR_NOMEM: return "out of memory";
        case MG_ERR_NOT_CONVERGED: return "not converged within max_iter";
        case MG_ERR_BREAKDOWN: return "Krylov breakdown (zero or non-finite scalar)";
        case MG_ERR_TIMEOUT: return "device wait timed out";
        case MG_ERR_UNSUPPORTED: return "unsupported request for this handle";
    }
    return "unknown status";
}

mg_status mg_setup(const mg_mesh* mesh, const mg_params* prm, const double* g, const mg_mixed* mixed,
                   mg_handle** out) {
    if (!out) return MG_ERR_ARG;
    *out = nullptr;
    TRY(mg_setup_check(mesh, prm, g, mixed));
    mg_handle* h = new (std::nothrow) mg_handle();
    if (!h) return MG_ERR_NOMEM;
    mg_status st = setup_impl(h, mesh, prm, g, mixed);
    if (st != MG_OK) {
        free_handle(h);
        return st;
    }
    *out = h;
    return MG_OK;
}

}  // extern "C"

static mg_status mg_setup_check(const mg_mesh* mesh, const mg_params* prm, const double* g, const mg_mixed* mixed) {
    if (!mesh || !prm || !g || !mesh->z_interfaces) return MG_ERR_ARG;
    if (mesh->n < 1 || mesh->nlev < 1 || mesh->nlev > MG_MAX_NLEV) return MG_ERR_ARG;
    if (!(mesh->radius > 0.0) || !(mesh->cs_dt > 0.0) || !std::isfinite(mesh->cs_dt)) return MG_ERR_ARG;
    if (prm->levels < 1 || prm->levels > MG_MAX_LEVELS) return MG_ERR_ARG;
    if (mesh->n % (1 << (prm->levels - 1)) != 0) return MG_ERR_ARG;
    if (!std::isfinite(prm->omega) || prm->n_pre < 0 || prm->n_post < 0 || prm->n_coarse < 1) return MG_ERR_ARG;
    if (prm->vcycle_precision < MG_FP64 || prm->vcycle_precision > MG_FP32_P64) return MG_ERR_ARG;
    if (prm->gcr_restart < 1 || prm->gcr_restart > MG_MAX_RESTART || prm->max_iter < 1) return MG_ERR_ARG;
    if (mixed && (!mixed->beta_up || !mixed->beta_dn || !std::isfinite(mixed->eps) || mixed->eps < 0.0 ||
                  (mixed->consistent != 0 && mixed->consistent != 1) || !std::isfinite(mixed->coriolis_f0) ||
                  std::fabs(mixed->coriolis_f0) >= 0.5))
        return MG_ERR_ARG;
    // the column kernels address a level with 32-bit offsets (horizontal faces: 2 kc)
    if (2.0 * (mesh->nlev + 1) * 6.0 * (double)mesh->n * mesh->n >= 4294967296.0) return MG_ERR_UNSUPPORTED;
    return MG_OK;
}

extern "C" {

mg_status mg_setup_9pt(const mg_mesh* mesh, const mg_params* prm, const double* g, double gamma2, mg_handle** out) {
    if (!out) return MG_ERR_ARG;
    *out = nullptr;
    if (!(gamma2 > 0.0) || !std::isfinite(gamma2) || !prm) return MG_ERR_ARG;
    if (prm->vcycle_precision == MG_FP32_BF16COEF || prm->vcycle_precision == MG_FP32_P64)
        return MG_ERR_UNSUPPORTED;
    if (!mesh || !g || !mesh->z_interfaces) return MG_ERR_ARG;
    mg_handle* h = nullptr;
    // validate exactly as mg_setup does, then build with the next-to-nearest fluxes
    TRY(mg_setup_check(mesh, prm, g, nullptr));
    h = new (std::nothrow) mg_handle();
    if (!h) return MG_ERR_NOMEM;
    const mg_status st = setup_impl(h, mesh, prm, g, nullptr, gamma2);
    if (st != MG_OK) {
        free_handle(h);
        return st;
    }
    *out = h;
    return MG_OK;
}

mg_status mg_setup_coeffs(const mg_mesh* mesh, const mg_params* prm, const double* coeffs, const double* cell_factors,
                          mg_handle** out) {
    if (!out) return MG_ERR_ARG;
    *out = nullptr;
    if (!coeffs) return MG_ERR_ARG;
    mg_handle* h = nullptr;
    TRY(mg_setup(mesh, prm, cell_factors, nullptr, &h));
    const size_t n6 = 6 * cells(h, 0);
    double* tmp = nullptr;
    mg_status st = MG_OK;
    if (!mem_alloc((void**)&tmp, n6 * sizeof(double), MEM_DEVICE)) {
        st = MG_ERR_NOMEM;
    } else if (cudaMemcpy(tmp, coeffs, n6 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        st = MG_ERR_CUDA;
    } else {
        st = set_coefficients_impl(h, tmp, nullptr);
        if (st == MG_OK && cudaDeviceSynchronize() != cudaSuccess) st = MG_ERR_CUDA;
    }
    mem_free(tmp, MEM_DEVICE);
    if (st != MG_OK) {
        mg_destroy(h);
        return st;
    }
    *out = h;
    return MG_OK;
}

mg_status mg_set_pressure_solver(mg_handle* h, const mg_pressure_solver* ps) {
    if (!h || !ps) return MG_ERR_ARG;
    if (ps->kind < MG_PS_MG || ps->kind > MG_PS_BICGSTAB_MG) return MG_ERR_ARG;
    const bool jac = ps->kind == MG_PS_JACOBI || ps->kind == MG_PS_BICGSTAB_JACOBI;
    const bool bicg = ps->kind == MG_PS_BICGSTAB_JACOBI || ps->kind == MG_PS_BICGSTAB_MG;
    if (jac && (ps->sweeps < 1 || !std::isfinite(ps->omega))) return MG_ERR_ARG;
    if (bicg && (!(ps->eps >= 0.0) || ps->max_iter < 1)) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    if (bicg && !h->bv[0]) {
        const size_t n = cells(h, 0);
        for (double*& v : h->bv) TRY(dalloc(h, &v, n));
    }
    CK(cudaDeviceSynchronize());
    h->ps = *ps;
    // the cached mixed-solve graphs hold the previous pressure solver
    for (int sys = 1; sys < 3; ++sys)
        for (cudaGraphExec_t& g : h->gexec[sys])
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    return MG_OK;
}

mg_status helmholtz_solve(mg_handle* h, const double* b, double* x, double* iterations, void* stream) {
    NvtxRange nvtx_("helmholtz_solve");
    if (!h || !b || !x || b == x) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    double it = 0.0;
    const mg_status st = run_pressure_solver(h, b, x, S(stream), &it);
    if (iterations) *iterations = it;
    return st;
}

mg_status mg_inner_stats(mg_handle* h, int64_t* solves, double* iterations) {
    if (!h) return MG_ERR_ARG;
    if (solves) *solves = h->ps_solves;
    if (iterations) *iterations = h->ps_iters;
    h->ps_solves = 0;
    h->ps_iters = 0.0;
    return MG_OK;
}

mg_status mg_set_coefficients(mg_handle* h, const double* coeffs, void* stream) {
    if (!h || !coeffs) return MG_ERR_ARG;
    if (h->mixed || h->nine) return MG_ERR_UNSUPPORTED;
    DeviceGuard dg(h->device);
    return set_coefficients_impl(h, coeffs, S(stream));
}

void mg_destroy(mg_handle* h) {
    if (!h) return;
    DeviceGuard dg(h->device);
    cudaDeviceSynchronize();
    free_handle(h);
}

mg_status mg_sizes(const mg_handle* h, int64_t* ncol, int64_t* ncell, int64_t* nu) {
    if (!h) return MG_ERR_ARG;
    if (ncol) *ncol = h->lv[0].ncol;
    if (ncell) *ncell = (int64_t)cells(h, 0);
    if (nu) *nu = h->nu;
    return MG_OK;
}

mg_status helmholtz_apply(mg_handle* h, const double* x, double* y, void* stream) {
    if (!h || !x || !y || x == y) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    if (h->nine) return launch_apply9(h, 0, x, y, S(stream));
    return launch_apply(h, 0, View<double, double>::lvl(h, 0), x, y, S(stream));
}

mg_status vcycle(mg_handle* h, const double* b, double* x, void* stream) {
    NvtxRange nvtx_("vcycle");
    if (!h || !b || !x || b == x) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    return run_vcycle(h, b, x, S(stream));
}

mg_status pressure_solve(mg_handle* h, const double* b, double* x, double tol, mg_solve_info* info,
                         void* stream) {
    NvtxRange nvtx_("pressure_solve");
    if (!h || !b || !x || b == x || !(tol >= 0.0)) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    auto A = [&](const double* z, double* w, int j, cudaStream_t q) { return apply_gcr(h, z, w, j, q); };
    auto P = [&](const double* r, double* z, cudaStream_t q) { return run_vcycle(h, r, z, q); };
    return gcr(h, 0, cells(h, 0), b, x, tol, info, s, A, P);
}

mg_status pressure_solve_adjoint(mg_handle* h, const double* g, double* lambda, double tol, mg_solve_info* info,
                                 void* stream) {
    NvtxRange nvtx_("pressure_solve_adjoint");
    if (!h || !g || !lambda || g == lambda || !(tol >= 0.0)) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    const int ncol = h->lv[0].ncol, nlev = h->nlev;
    const size_t n = cells(h, 0);
    const dim3 grid((ncol + 127) / 128, nlev);
    // H^T = V H V^-1 (V H is symmetric): lambda = V H^-1 (V^-1 g)
    {
        Prof pr(h, MG_K_DOT, 0, 16.0 * n, s);
        mg::k_scale_volume<<<grid, 128, 0, s>>>(ncol, nlev, h->area0, h->dz, g, h->adj, false);
        CK(cudaGetLastError());
    }
    auto A = [&](const double* z, double* w, int j, cudaStream_t q) { return apply_gcr(h, z, w, j, q); };
    auto P = [&](const double* r, double* z, cudaStream_t q) { return run_vcycle(h, r, z, q); };
    const mg_status st = gcr(h, 0, n, h->adj, lambda, tol, info, s, A, P);
    if (st == MG_OK || st == MG_ERR_NOT_CONVERGED) {
        Prof pr(h, MG_K_DOT, 0, 16.0 * n, s);
        mg::k_scale_volume<<<grid, 128, 0, s>>>(ncol, nlev, h->area0, h->dz, lambda, lambda, true);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
    }
    return st;
}

mg_status helmholtz_coefficient_gradient(mg_handle* h, const double* lambda, const double* x, double* grad,
                                         void* stream) {
    if (!h || !lambda || !x || !grad) return MG_ERR_ARG;
    if (h->nine) return MG_ERR_UNSUPPORTED;
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    const Lvl<double, double> L = View<double, double>::lvl(h, 0);
    Prof pr(h, MG_K_DOT, 0, 64.0 * cells(h, 0), s);   // lambda, x (read), 6 gradients (written)
    mg::k_coef_grad<<<dim3((L.ncol + 127) / 128, L.nlev), 128, 0, s>>>(L, lambda, x, grad);
    CK(cudaGetLastError());
    return MG_OK;
}

mg_status ensemble_pressure_solve(mg_handle* const* handles, int32_t count, const double* const* b,
                                  double* const* x, double tol, mg_solve_info* infos, int32_t* statuses,
                                  void* stream) {
    NvtxRange nvtx_("ensemble_pressure_solve");
    if (count < 0 || (count > 0 && (!handles || !b || !x)) || !(tol >= 0.0)) return MG_ERR_ARG;
    if (count == 0) return MG_OK;
    for (int i = 0; i < count; ++i) {
        if (!handles[i] || !b[i] || !x[i] || b[i] == x[i] || handles[i]->device != handles[0]->device)
            return MG_ERR_ARG;
        for (int k = 0; k < i; ++k)
            if (handles[k] == handles[i]) return MG_ERR_ARG;   // a handle holds one solve's workspace
    }
    DeviceGuard dg(handles[0]->device);
    // every member starts after the work already queued on the caller's stream
    CK(cudaEventRecord(handles[0]->evx, S(stream)));
    std::vector<GcrRun> g(count);
    for (int i = 0; i < count; ++i) {
        mg_handle* h = handles[i];
        g[i].sys = 0;
        g[i].n = cells(h, 0);
        g[i].x = x[i];
        g[i].tol = tol;
        CK(cudaStreamWaitEvent(h->run, handles[0]->evx, 0));
        TRY(gcr_start(h, g[i], b[i], h->run));
    }
    for (int i = 0; i < count; ++i) {
        CK(cudaStreamSynchronize(handles[i]->run));
        gcr_started(handles[i], g[i]);
    }
    // rounds: every unfinished member launches one iteration on its stream (the members run
    // side by side on the GPU), then the host collects the residual norms
    for (bool any = true; any;) {
        any = false;
        for (int i = 0; i < count; ++i) {
            if (!g[i].active) continue;
            mg_handle* h = handles[i];
            auto A = [h](const double* z, double* w, int j, cudaStream_t q) { return apply_gcr(h, z, w, j, q); };
            auto P = [h](const double* r, double* z, cudaStream_t q) { return run_vcycle(h, r, z, q); };
            TRY(gcr_launch(h, g[i], h->run, A, P));
        }
        for (int i = 0; i < count; ++i) {
            if (!g[i].active) continue;
            CK(cudaStreamSynchronize(handles[i]->run));
            TRY(gcr_landed(handles[i], g[i], handles[i]->run));
            any = any || g[i].active;
        }
    }
    mg_status st = MG_OK;
    for (int i = 0; i < count; ++i) CK(cudaEventRecord(handles[i]->ev1, handles[i]->run));
    for (int i = 0; i < count; ++i) {
        CK(cudaEventSynchronize(handles[i]->ev1));
        gcr_info(handles[i], g[i], infos ? infos + i : nullptr);
        if (statuses) statuses[i] = g[i].st;
        if (st == MG_OK) st = g[i].st;
    }
    return st;
}

mg_status mg_ensemble_create(mg_handle* const* handles, int32_t count, const double* const* b, double* const* x,
                             double tol, mg_ensemble** out) {
    if (!out) return MG_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !handles || !b || !x || !(tol >= 0.0)) return MG_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        if (!handles[i] || !b[i] || !x[i] || b[i] == x[i] || handles[i]->device != handles[0]->device)
            return MG_ERR_ARG;
        for (int k = 0; k < i; ++k)
            if (handles[k] == handles[i]) return MG_ERR_ARG;
        if (handles[i]->prof || handles[i]->mixed) return MG_ERR_UNSUPPORTED;
    }
    DeviceGuard dg(handles[0]->device);
    mg_ensemble* e = new (std::nothrow) mg_ensemble();
    if (!e) return MG_ERR_NOMEM;
    e->device = handles[0]->device;
    e->count = count;
    e->hs.assign(handles, handles + count);
    const mg_status st = build_ensemble(e, b, x, tol);
    if (st != MG_OK) {
        cudaStreamCaptureStatus cst;
        if (e->cs && cudaStreamIsCapturing(e->cs, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(e->cs, &g);
        }
        cudaGetLastError();
        free_ensemble(e);
        return st;
    }
    *out = e;
    return MG_OK;
}

mg_status mg_ensemble_solve(mg_ensemble* e, mg_solve_info* infos, int32_t* statuses, void* stream) {
    NvtxRange nvtx_("mg_ensemble_solve");
    if (!e) return MG_ERR_ARG;
    DeviceGuard dg(e->device);
    cudaStream_t s = S(stream);
    CK(cudaGraphLaunch(e->exec, s));
    CK(cudaStreamSynchronize(s));
    mg_status st = MG_OK;
    for (int i = 0; i < e->count; ++i) {
        const mg::EnsState& m = e->host_st[i];
        if (infos) {
            infos[i].iters = m.it;
            infos[i].rel_res = m.rel;
            infos[i].ms = 1e-6 * (double)(e->host_stamps[1 + i] - e->host_stamps[0]);
        }
        if (statuses) statuses[i] = m.status;
        if (st == MG_OK) st = (mg_status)m.status;
    }
    return st;
}

void mg_ensemble_destroy(mg_ensemble* e) {
    if (!e) return;
    DeviceGuard dg(e->device);
    cudaDeviceSynchronize();
    free_ensemble(e);
}

mg_status mixed_solve(mg_handle* h, const double* rhs_u, const double* rhs_p, double* u, double* p, double tol,
                      mg_solve_info* info, void* stream) {
    NvtxRange nvtx_("mixed_solve");
    if (!h || !rhs_u || !rhs_p || !u || !p || !(tol >= 0.0)) return MG_ERR_ARG;
    if (!h->mixed) return MG_ERR_UNSUPPORTED;
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    const size_t nu = (size_t)h->nu, np = cells(h, 0), n = nu + np;
    // GCR runs on concatenated [u; p] vectors held by the handle
    CK(cudaMemcpyAsync(h->mb, rhs_u, nu * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->mb + nu, rhs_p, np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    auto A = [&](const double* v, double* y, int j, cudaStream_t q) {
        TRY(mixed_apply_impl(h, v, v + nu, y, y + nu, q));
        return gcr_sums(h, n, y, j, q);
    };
    auto P = [&](const double* r, double* z, cudaStream_t q) { return schur_impl(h, r, r + nu, z, z + nu, q); };
    const mg_status st = gcr(h, 1, n, h->mb, h->mx, tol, info, s, A, P);
    if (st == MG_OK || st == MG_ERR_NOT_CONVERGED || st == MG_ERR_BREAKDOWN) {
        CK(cudaMemcpyAsync(u, h->mx, nu * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(p, h->mx + nu, np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    return st;
}

mg_status mixed_solve_adjoint(mg_handle* h, const double* g_u, const double* g_p, double* lam_u, double* lam_p,
                              double tol, mg_solve_info* info, void* stream) {
    NvtxRange nvtx_("mixed_solve_adjoint");
    if (!h || !g_u || !g_p || !lam_u || !lam_p || !(tol >= 0.0)) return MG_ERR_ARG;
    if (!h->mixed) return MG_ERR_UNSUPPORTED;
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    const size_t nu = (size_t)h->nu, np = cells(h, 0), n = nu + np;
    // A^T = S J A-hat J S^-1: lambda = S J A-hat^-1 (J S^-1 g), A-hat preconditioned by the
    // Schur-complement step of A itself (its transpose is S J P J S^-1 as well)
    TRY(mixed_adj_scale<false>(h, g_u, g_p, h->mb, h->mb + nu, s));
    auto A = [&](const double* v, double* y, int j, cudaStream_t q) {
        TRY(mixed_apply_hat_impl(h, v, v + nu, y, y + nu, q));
        return gcr_sums(h, n, y, j, q);
    };
    auto P = [&](const double* r, double* z, cudaStream_t q) { return schur_impl(h, r, r + nu, z, z + nu, q); };
    const mg_status st = gcr(h, 2, n, h->mb, h->mx, tol, info, s, A, P);
    if (st == MG_OK || st == MG_ERR_NOT_CONVERGED || st == MG_ERR_BREAKDOWN) {
        TRY(mixed_adj_scale<true>(h, h->mx, h->mx + nu, lam_u, lam_p, s));
        CK(cudaStreamSynchronize(s));
    }
    return st;
}

mg_status mixed_coefficient_gradient(mg_handle* h, const double* lam_u, const double* u, const double* p,
                                     double* grad_g, double* grad_beta_up, double* grad_beta_dn, void* stream) {
    if (!h || !lam_u || !u || !p || !grad_g || !grad_beta_up || !grad_beta_dn) return MG_ERR_ARG;
    if (!h->mixed) return MG_ERR_UNSUPPORTED;
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    const mg::MixedDev& M = h->md;
    const size_t nh = (size_t)M.nlev * M.nfh;
    const int bd = 128;
    Prof pr(h, MG_K_DOT, 0, 8.0 * (3.0 * h->nu + 2.0 * cells(h, 0)), s, 3);
    mg::k_mx_grad_g<<<dim3((M.ncol + bd - 1) / bd, M.nlev), bd, 0, s>>>(M, lam_u, p, grad_g);
    mg::k_mx_grad_beta<<<dim3((M.ncol + bd - 1) / bd, M.nlev + 1), bd, 0, s>>>(M, lam_u + nh, u + nh, grad_beta_up,
                                                                              grad_beta_dn);
    CK(cudaGetLastError());
    return MG_OK;
}

mg_status mixed_apply_transpose(mg_handle* h, const double* u, const double* p, double* yu, double* yp,
                                void* stream) {
    if (!h || !u || !p || !yu || !yp || u == yu || p == yp) return MG_ERR_ARG;
    if (!h->mixed) return MG_ERR_UNSUPPORTED;
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    const size_t nu = (size_t)h->nu;
    TRY(mixed_adj_scale<false>(h, u, p, h->mb, h->mb + nu, s));
    TRY(mixed_apply_hat_impl(h, h->mb, h->mb + nu, h->mx, h->mx + nu, s));
    return mixed_adj_scale<true>(h, h->mx, h->mx + nu, yu, yp, s);
}

mg_status mg_level_apply(mg_handle* h, int32_t level, const double* x, double* y, void* stream) {
    TRY(check_level(h, level));
    if (!x || !y || x == y) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    if (h->nine) return launch_apply9(h, level, x, y, S(stream));
    return launch_apply(h, level, View<double, double>::lvl(h, level), x, y, S(stream));
}

mg_status mg_smooth(mg_handle* h, int32_t level, const double* b, const double* x_in, double* x_out,
                    int32_t sweeps, void* stream) {
    TRY(check_level(h, level));
    if (!b || !x_out || sweeps < 0 || b == x_out) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    DevLevel& d = h->lv[level];
    const Lvl<double, double> L = View<double, double>::lvl(h, level);
    const size_t n = cells(h, level);
    const double* cur = x_in;
    for (int i = 0; i < sweeps; ++i) {
        double* dst = (cur == d.x64[0]) ? d.x64[1] : d.x64[0];
        if (h->nine) TRY((sweep9<double, double, double>(h, level, cur, b, dst, h->prm.omega, s)));
        else TRY((sweep_any<double, double, double, double>(h, level, L, cur, (const double*)nullptr, 0, b, nullptr,
                                                            dst, h->prm.omega, s)));
        cur = dst;
    }
    if (cur == nullptr) CK(cudaMemsetAsync(x_out, 0, n * sizeof(double), s));
    else if (cur != x_out) CK(cudaMemcpyAsync(x_out, cur, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return MG_OK;
}

mg_status mg_residual_restrict(mg_handle* h, int32_t level, const double* b, const double* x, double* bc,
                               void* stream) {
    TRY(check_level(h, level));
    if (level + 1 >= h->L || !b || !x || !bc) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    if (h->nine) return restrict9<double, double, double>(h, level, x, b, bc, S(stream));
    return launch_restrict<double, double, false, double, double, double>(
        h, level, View<double, double>::lvl(h, level), x, b, h->lv[level].w64, bc, h->lv[level + 1].ncol, S(stream));
}

mg_status mg_prolong_add(mg_handle* h, int32_t level, const double* xc, double* x, void* stream) {
    TRY(check_level(h, level));
    if (level + 1 >= h->L || !xc || !x) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    const DevLevel& d = h->lv[level];
    return launch_prolong<double, false, double, double>(h, level, d.n, d.ncol, h->lv[level + 1].ncol, h->nlev, x, xc, x,
                                                         S(stream));
}

mg_status mixed_apply(mg_handle* h, const double* u, const double* p, double* yu, double* yp, void* stream) {
    if (!h || !u || !p || !yu || !yp) return MG_ERR_ARG;
    if (!h->mixed) return MG_ERR_UNSUPPORTED;
    DeviceGuard dg(h->device);
    return mixed_apply_impl(h, u, p, yu, yp, S(stream));
}

mg_status schur_precond(mg_handle* h, const double* ru, const double* rp, double* u, double* p, void* stream) {
    if (!h || !ru || !rp || !u || !p) return MG_ERR_ARG;
    if (!h->mixed) return MG_ERR_UNSUPPORTED;
    DeviceGuard dg(h->device);
    return schur_impl(h, ru, rp, u, p, S(stream));
}

mg_status mg_autotune(mg_handle* h, int32_t* choices, void* stream) {
    NvtxRange nvtx_("mg_autotune");
    if (!h) return MG_ERR_ARG;
    if (h->prof || h->nine) return MG_ERR_UNSUPPORTED;   // the tuner uses the per-launch profiler itself
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    const int L = h->L;
    const size_t N = cells(h, 0);
    constexpr int REPS = 3;
    // every launch of REPS V-cycles is recorded: 2 kinds x L levels x (sweeps + 1) at most
    const int cap = 2 * REPS * L * (h->prm.n_pre + h->prm.n_post + h->prm.n_coarse + 4);
    while ((int)h->evpool.size() < 2 * cap) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        h->evpool.push_back(e);
    }
    // a V-cycle on the handle's own buffers: b = 0 (the launches, and so their times, do not
    // depend on the values)
    CK(cudaMemsetAsync(h->r, 0, N * sizeof(double), s));
    std::vector<double> sweep_ms(L), restr_ms(L);
    auto measure = [&]() -> mg_status {
        TRY(run_vcycle(h, h->r, h->adj, s));   // warm-up with this shape
        h->prof_kind = -1;
        h->prof_level = -1;
        h->recs.clear();
        h->prof = true;
        mg_status st = MG_OK;
        for (int i = 0; i < REPS && st == MG_OK; ++i) st = run_vcycle(h, h->r, h->adj, s);
        h->prof = false;
        TRY(st);
        CK(cudaStreamSynchronize(s));
        std::fill(sweep_ms.begin(), sweep_ms.end(), 0.0);
        std::fill(restr_ms.begin(), restr_ms.end(), 0.0);
        for (size_t i = 0; i < h->recs.size(); ++i) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, h->evpool[2 * i], h->evpool[2 * i + 1]));
            const auto& r = h->recs[i];
            if (r.level < 0 || r.level >= L) continue;
            if (r.kind == MG_K_SWEEP) sweep_ms[r.level] += ms;
            if (r.kind == MG_K_RESTRICT) restr_ms[r.level] += ms;
        }
        h->recs.clear();
        return MG_OK;
    };
    // sweep blocks: 64 or 128 threads (two warps hold the two halves of 32 columns; the
    // kernel's launch bounds allow 128)
    std::vector<int> best_bd(L, 0);
    std::vector<double> best_t(L, 1e300);
    for (int bd : {64, 128}) {
        for (int l = 0; l < L; ++l) h->lv[l].sweep_bd = bd;
        TRY(measure());
        for (int l = 0; l < L; ++l)
            if (sweep_ms[l] < best_t[l]) best_t[l] = sweep_ms[l], best_bd[l] = bd;
    }
    for (int l = 0; l < L; ++l) h->lv[l].sweep_bd = best_bd[l];
    // residual + restriction: levels per thread, copy ring or register ring
    std::vector<int> best_kc(L, 0), best_as(L, -1);
    std::fill(best_t.begin(), best_t.end(), 1e300);
    for (int as : {0, 1})
        for (int kc : {4, 8, 16, 24, 35, 70}) {
            for (int l = 0; l < L; ++l) h->lv[l].restrict_kc = kc, h->lv[l].restrict_async = as;
            TRY(measure());
            for (int l = 0; l + 1 < L; ++l)
                if (restr_ms[l] < best_t[l]) best_t[l] = restr_ms[l], best_kc[l] = kc, best_as[l] = as;
        }
    for (int l = 0; l < L; ++l) h->lv[l].restrict_kc = best_kc[l], h->lv[l].restrict_async = best_as[l];
    // the cached GCR graphs hold the old launch shapes
    for (auto& row : h->gexec)
        for (cudaGraphExec_t& g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    if (choices)
        for (int l = 0; l < L; ++l) {
            choices[3 * l] = best_bd[l];
            choices[3 * l + 1] = best_kc[l];
            choices[3 * l + 2] = best_as[l];
        }
    return MG_OK;
}

mg_status mg_profile_start(mg_handle* h, int32_t capacity, int32_t kind, int32_t level) {
    if (!h || capacity < 1 || capacity > (1 << 20)) return MG_ERR_ARG;
    h->prof_kind = kind < 0 ? -1 : kind;
    h->prof_level = level < 0 ? -1 : level;
    DeviceGuard dg(h->device);
    while ((int)h->evpool.size() < 2 * capacity) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        h->evpool.push_back(e);
    }
    h->recs.clear();
    h->recs.reserve(capacity);
    h->prof = true;
    return MG_OK;
}

mg_status mg_profile_stop(mg_handle* h, mg_kernel_record* out, int32_t cap, int32_t* count) {
    if (!h || !count || (cap > 0 && !out)) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    h->prof = false;
    CK(cudaDeviceSynchronize());
    const int n = (int)h->recs.size();
    for (int i = 0; i < n && i < cap; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->evpool[2 * i], h->evpool[2 * i + 1]));
        out[i].kind = h->recs[i].kind;
        out[i].level = h->recs[i].level;
        out[i].variant = h->recs[i].variant;
        out[i].bytes = h->recs[i].bytes;
        out[i].ms = ms;
    }
    *count = n;
    h->recs.clear();
    return MG_OK;
}

}  // extern "C"

// =====================================================================================
// Block-Jacobi smoothing without allocation (see mg_smooth_noalloc in mgsolve.h).
//
// The intermediate iterates that mg_smooth keeps in the handle's workspace live here in
// one fixed device array instead.  Every GPU that loads this library holds the array until
// the process exits, and every call shares it.
static __device__ __align__(256) double g_smooth_scratch[MG_NOALLOC_MAX_CELLS];

namespace {
// Host code cannot use g_smooth_scratch as a device address: on the host it names a
// stand-in object.  Its device address is looked up once per device (with that device
// current) and kept here.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double* g_scratch_addr[kMaxDevices] = {};

mg_status scratch_address(int device, double** out) {
    if (device < 0 || device >= kMaxDevices) return MG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_smooth_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return MG_ERR_CUDA;
        }
        g_scratch_addr[device] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[device];
    return MG_OK;
}
}  // namespace

extern "C" mg_status mg_smooth_noalloc(mg_handle* h, int32_t level, const double* b, const double* x_in,
                                       double* x_out, int32_t sweeps, void* stream) {
    TRY(check_level(h, level));
    if (!b || !x_out || sweeps < 0 || b == x_out) return MG_ERR_ARG;
    if (h->nine) return MG_ERR_UNSUPPORTED;
    const size_t n = cells(h, level);
    if (n > (size_t)MG_NOALLOC_MAX_CELLS) return MG_ERR_ARG;
    DeviceGuard dg(h->device);
    double* scratch = nullptr;
    TRY(scratch_address(h->device, &scratch));
    cudaStream_t s = S(stream);
    const Lvl<double, double> L = View<double, double>::lvl(h, level);
    if (sweeps == 0) {
        if (!x_in) CK(cudaMemsetAsync(x_out, 0, n * sizeof(double), s));
        else if (x_in != x_out) CK(cudaMemcpyAsync(x_out, x_in, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        return MG_OK;
    }
    // Sweeps alternate between the scratch array and x_out, ordered so that the last one
    // writes x_out.  A sweep never writes the array it reads, so when x_in aliases x_out
    // and x_out would be the first target, the first sweep goes to the scratch array and
    // the result is copied to x_out at the end.
    bool to_out = ((sweeps - 1) % 2) == 0;
    const bool copy_back = to_out && x_in == x_out;
    if (copy_back) to_out = false;
    const double* cur = x_in;
    for (int i = 0; i < sweeps; ++i) {
        double* dst = to_out ? x_out : scratch;
        TRY((sweep_any<double, double, double, double>(nullptr, level, L, cur, (const double*)nullptr, 0, b,
                                                       nullptr, dst, h->prm.omega, s)));
        cur = dst;
        to_out = !to_out;
    }
    if (cur != x_out) CK(cudaMemcpyAsync(x_out, cur, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return MG_OK;
}
