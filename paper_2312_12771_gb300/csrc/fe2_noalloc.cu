// fe2_rve_solve_noalloc: the fused RVE solve for callers that cannot allocate
// device memory.
//
// Callers such as code running inside another framework's memory pool, a
// plugin or extension whose host forbids cudaMalloc / cudaFree while it owns
// the device, or real-time code that must not touch the allocator once started,
// cannot use the context API: a context allocates its RVE state and its
// factorisation workspace.  This entry point takes every input and output as a
// caller-owned device pointer and keeps all intermediate data (descriptors,
// neighbour table, reduced operators, band factor, solutions, residuals) in
// one file-scope __device__ array of FE2_NOALLOC_SCRATCH_BYTES.  The array
// exists on every GPU that loads this library, for the life of the process.
//
// It runs the same kernels as fe2_rve_solve on the mixed path (general
// assembly kernel for both material models, FP32 band factor, FP64 residual,
// residual-corrected Schur complement, no refinement sweeps).  Until one call
// on a device has passed it, every call reads back what the set-up kernel
// wrote and checks every address and index the solve kernels take from it
// before launching them; failures leave a reason for fe2_noalloc_last_error.
// The inputs live on the device, so a small kernel validates them there: an
// RVE with a phase index >= nphase or an unknown material model gets
// rve_status FE2_ERR_ARG, and its descriptor is pointed at a single-phase
// linear material in the scratch array so that no kernel reads outside the
// caller's arrays; its outputs are then meaningless.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fe2_internal.cuh"

using namespace fe2;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FE2_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};   // device address of the array, per device
bool g_verified[kMaxDevices] = {false};          // a call on the device passed the set-up read-back
char g_err[256] = "";                            // reason of the last failed call

fe2_status fail_msg(fe2_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NoallocLayout {
    int N, nn, nm, kd, nmp, nr;
    size_t off_desc, off_ids, off_tol, off_nbr, off_safe, off_rve, rve_stride, off_ws, ws_stride, offY, offR, offD,
        total;
    size_t o_st, o_rhs, o_X, o_mm;
};

NoallocLayout layout_for(int N, int n) {
    NoallocLayout L{};
    L.N = N;
    L.nn = N * N;
    L.nm = 2 * (L.nn - 1);
    int kd = 4 * N + 5;  // half bandwidth of the folded periodic ordering (2D)
    kd = kd < NB ? NB : kd;
    L.kd = kd;
    L.nmp = (L.nm + NB - 1) / NB * NB;
    L.nr = 5;
    size_t o = 0;
    L.off_desc = o;
    o += a256(sizeof(RveDev) * (size_t)n);
    L.off_ids = o;
    o += a256(sizeof(int) * (size_t)n);
    L.off_tol = o;
    o += 256;
    L.off_nbr = o;
    o += a256(sizeof(int) * 9 * (size_t)L.nn);
    L.off_safe = o;  // stand-in inputs of a rejected RVE: one linear material, phase 0 everywhere
    o += a256(4 * sizeof(double) + (size_t)L.nn);
    // per-RVE reduced operators and solutions
    L.o_st = 0;
    size_t r = a256(36 * (size_t)L.nn * 8);
    L.o_rhs = r;
    r += a256((size_t)L.nr * L.nm * 8);
    L.o_X = r;
    r += a256((size_t)L.nr * L.nm * 8);
    L.o_mm = r;
    r += a256(20 * 8);
    L.rve_stride = r;
    L.off_rve = o;
    o += r * (size_t)n;
    // factorisation workspace (FP32 band factor)
    size_t w = a256((size_t)L.nmp * (L.kd + 1) * 4);
    L.offY = w;
    w += a256((size_t)L.nr * L.nmp * 4);
    L.offR = w;
    w += a256((size_t)L.nr * L.nm * 8);
    L.offD = w;
    w += a256((size_t)L.nmp * 4);
    L.ws_stride = w;
    L.off_ws = o;
    o += w * (size_t)n;
    L.total = o;
    return L;
}

// Descriptors, ids, tolerance and the folded-ordering neighbour table, written
// into the scratch array by the device itself (nothing is copied from the host).
__global__ void k_noalloc_setup(unsigned char* base, NoallocLayout L, int n, int nphase,
                                const uint8_t* __restrict__ phase, const double* __restrict__ mat, double tol) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    RveDev* desc = (RveDev*)(base + L.off_desc);
    int* ids = (int*)(base + L.off_ids);
    int* nbr = (int*)(base + L.off_nbr);
    const int N = L.N;
    if (t < n) {
        // every field is stored in place: nvcc 13.0 compiled a whole-struct copy of a
        // local descriptor here into a copy of the equally sized (152-byte) layout
        // parameter L, which the host's first-call read-back (check_setup) exposed
        unsigned char* rb = base + L.off_rve + L.rve_stride * t;
        RveDev* r = desc + t;
        r->N = N;
        r->d = 2;
        r->nm = L.nm;
        r->kd = L.kd;
        r->nn = L.nn;
        r->nphase = nphase;
        r->nm_pad = L.nmp;
        r->nr = L.nr;
        r->phase = phase + (size_t)t * L.nn;
        r->mat = mat + (size_t)t * nphase * 4;
        r->w = nullptr;
        r->stencil = (double*)(rb + L.o_st);
        r->rhs = (double*)(rb + L.o_rhs);
        r->X = (double*)(rb + L.o_X);
        r->KMM = (double*)(rb + L.o_mm);
        r->Pint = (double*)(rb + L.o_mm) + 16;
        r->elem = nullptr;
        r->nbr = nbr;
        r->zero_w = 1;
        r->nq = 1;
        for (int g = 0; g < 4; ++g) r->wq[g] = g == 0 ? 1.0 : 0.0;
        ids[t] = t;
    }
    if (t == 0) {
        double* sm = (double*)(base + L.off_safe);
        sm[0] = FE2_MODEL_LINEAR, sm[1] = 1.0, sm[2] = 0.3, sm[3] = 0.0;
        *(double*)(base + L.off_tol) = tol;
        // the kernel's view of the layout and of the descriptor size, for the host's first-call check
        int* v = (int*)(base + L.off_tol + 16);
        v[0] = L.N, v[1] = L.nn, v[2] = L.nm, v[3] = L.kd, v[4] = L.nmp, v[5] = L.nr;
        v[6] = (int)sizeof(RveDev), v[7] = (int)sizeof(NoallocLayout);
    }
    uint8_t* sp = base + L.off_safe + 4 * sizeof(double);
    for (int k = t; k < L.nn; k += gridDim.x * blockDim.x) sp[k] = 0;
    for (int k = t; k < L.nn * 9; k += gridDim.x * blockDim.x) {
        const int q = k / 9, off = k - 9 * q;
        const int i = unfold_pos(q % N, N), j = unfold_pos(q / N, N);
        const int dx = off % 3 - 1, dy = off / 3 - 1;
        nbr[k] = fold_pos((i + dx + N) % N, N) + N * fold_pos((j + dy + N) % N, N);
    }
}

// One CTA per RVE: every phase byte below nphase, every material model known
// (its parameters finite).  A rejected RVE keeps FE2_ERR_ARG in rve_status
// (the later kernels only overwrite FE2_OK) and reads the stand-in inputs.
__global__ void k_noalloc_validate(unsigned char* base, NoallocLayout L, int nphase, const uint8_t* __restrict__ phase,
                                   const double* __restrict__ mat, int* __restrict__ status) {
    const int t = blockIdx.x;
    int bad = 0;
    const uint8_t* ph = phase + (size_t)t * L.nn;
    for (int k = threadIdx.x; k < L.nn; k += blockDim.x) bad |= ph[k] >= nphase;
    if (threadIdx.x < nphase) {
        const double* m = mat + ((size_t)t * nphase + threadIdx.x) * 4;
        const double model = m[0];
        bad |= !(model == FE2_MODEL_LINEAR || model == FE2_MODEL_NEOHOOKE || model == FE2_MODEL_MOONEY_RIVLIN);
        bad |= !(isfinite(m[1]) && isfinite(m[2]) && isfinite(m[3]));
    }
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0) {
        RveDev* r = (RveDev*)(base + L.off_desc) + t;
        r->mat = (const double*)(base + L.off_safe);
        r->phase = base + L.off_safe + 4 * sizeof(double);
        r->nphase = 1;
        status[t] = FE2_ERR_ARG;
    }
}

// Host check of what k_noalloc_setup wrote (one synchronising read-back).
fe2_status check_setup(const unsigned char* base, const NoallocLayout& L, int n, int nphase, const uint8_t* phase,
                       const double* mat, cudaStream_t s) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_msg(FE2_ERR_CUDA, "set-up kernel: %s", cudaGetErrorString(e));
    std::vector<RveDev> desc((size_t)n);
    std::vector<int> ids((size_t)n), nbr((size_t)L.nn * 9);
    int v[8];
    if ((e = cudaMemcpy(v, base + L.off_tol + 16, sizeof(v), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(desc.data(), base + L.off_desc, sizeof(RveDev) * n, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(ids.data(), base + L.off_ids, sizeof(int) * n, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(nbr.data(), base + L.off_nbr, sizeof(int) * nbr.size(), cudaMemcpyDeviceToHost)) !=
            cudaSuccess)
        return fail_msg(FE2_ERR_CUDA, "read-back of the set-up: %s", cudaGetErrorString(e));
    if (v[0] != L.N || v[1] != L.nn || v[2] != L.nm || v[3] != L.kd || v[4] != L.nmp || v[5] != L.nr ||
        v[6] != (int)sizeof(RveDev) || v[7] != (int)sizeof(NoallocLayout))
        return fail_msg(FE2_ERR_CUDA,
                        "set-up kernel saw N=%d nn=%d nm=%d kd=%d nmp=%d nr=%d sizes %d %d (host %d %d %d %d %d %d "
                        "sizes %d %d)",
                        v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], L.N, L.nn, L.nm, L.kd, L.nmp, L.nr,
                        (int)sizeof(RveDev), (int)sizeof(NoallocLayout));
    for (int t = 0; t < n; ++t) {
        const RveDev& r = desc[t];
        const unsigned char* rb = base + L.off_rve + L.rve_stride * t;
        const struct {
            bool ok;
            const char* what;
        } c[] = {{ids[t] == t, "id"},
                 {r.N == L.N && r.d == 2 && r.nm == L.nm && r.kd == L.kd && r.nn == L.nn, "sizes"},
                 {r.nphase == nphase && r.nm_pad == L.nmp && r.nr == L.nr, "phases/padding/rhs"},
                 {r.zero_w == 1 && !r.w && !r.elem, "w/elem"},
                 {r.phase == phase + (size_t)t * L.nn && r.mat == mat + (size_t)t * nphase * 4, "phase/mat"},
                 {(const unsigned char*)r.stencil == rb + L.o_st && (const unsigned char*)r.rhs == rb + L.o_rhs &&
                      (const unsigned char*)r.X == rb + L.o_X,
                  "stencil/rhs/X"},
                 {(const unsigned char*)r.KMM == rb + L.o_mm && r.Pint == r.KMM + 16, "KMM/Pint"},
                 {(const unsigned char*)r.nbr == base + L.off_nbr, "nbr"}};
        for (const auto& x : c)
            if (!x.ok)
                return fail_msg(FE2_ERR_CUDA,
                                "set-up descriptor %d: %s not as written (N=%d d=%d nm=%d kd=%d nn=%d nphase=%d "
                                "nm_pad=%d nr=%d zero_w=%d nq=%d)",
                                t, x.what, r.N, r.d, r.nm, r.kd, r.nn, r.nphase, r.nm_pad, r.nr, r.zero_w, r.nq);
    }
    for (size_t k = 0; k < nbr.size(); ++k)
        if (nbr[k] < 0 || nbr[k] >= L.nn)
            return fail_msg(FE2_ERR_CUDA, "set-up neighbour table entry %zu = %d out of range", k, nbr[k]);
    return FE2_OK;
}

}  // namespace

extern "C" fe2_status fe2_rve_solve_noalloc(int N, int n, int nphase, const uint8_t* phase, const double* mat,
                                            const double* Fbar, double* sigma_eff, double* Cbar, int* rve_status,
                                            double* err_est, void* cuda_stream) {
    g_err[0] = '\0';
    if (N < 3 || n < 1 || nphase < 1 || nphase > MAX_PHASES)
        return fail_msg(FE2_ERR_ARG, "sizes out of range (N=%d n=%d nphase=%d)", N, n, nphase);
    if (!phase || !mat || !Fbar || !sigma_eff || !Cbar || !rve_status) return fail_msg(FE2_ERR_ARG, "NULL pointer");
    const NoallocLayout L = layout_for(N, n);
    if (L.kd + L.nr + 32 > FACT_THREADS) return fail_msg(FE2_ERR_ARG, "N=%d: band too wide", N);
    if (L.total > (size_t)FE2_NOALLOC_SCRATCH_BYTES)  // beyond the fixed scratch
        return fail_msg(FE2_ERR_BUDGET, "%zu bytes exceed the scratch array", L.total);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail_msg(FE2_ERR_CUDA, "no usable current device");
    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return fail_msg(FE2_ERR_CUDA, "device attribute query failed");
    if ((int)factor_smem_bytes(L.kd, L.nr, false) > smem_optin)
        return fail_msg(FE2_ERR_ARG, "N=%d: factor window exceeds shared memory", N);
    // one-time set-up per device (with that device current): the device address
    // of the scratch array; host code must not use the symbol itself
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return fail_msg(FE2_ERR_CUDA, "scratch address: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    unsigned char* base = (unsigned char*)g_scratch_addr[dev];
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int setup_threads = 256;
    const int setup_blocks = (n > L.nn * 9 ? n : L.nn * 9) / setup_threads + 1;
    k_noalloc_setup<<<setup_blocks, setup_threads, 0, s>>>(base, L, n, nphase, phase, mat, 1e-10);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return fail_msg(FE2_ERR_CUDA, "set-up launch: %s", cudaGetErrorString(le));
    // until a call on this device has passed it: read the descriptors, ids and
    // neighbour table back and confirm every address and index the solve kernels
    // derive from them (a failed check is repeated by the next call)
    if (!g_verified[dev]) {
        const fe2_status st = check_setup(base, L, n, nphase, phase, mat, s);
        if (st != FE2_OK) return st;
        g_verified[dev] = true;
    }
    const RveDev* tab = (const RveDev*)(base + L.off_desc);
    const int* ids = (const int*)(base + L.off_ids);
    const double* tol = (const double*)(base + L.off_tol);
    Workspace ws{(char*)base + L.off_ws, L.ws_stride, L.offY, L.offR, L.offD, 0};
    cudaError_t e;
#define NOALLOC_STEP(what, call) \
    if ((e = (call)) != cudaSuccess) return fail_msg(FE2_ERR_CUDA, "%s launch: %s", what, cudaGetErrorString(e))
    NOALLOC_STEP("check", launch_check_fbar(Fbar, n, 2, rve_status, s));
    k_noalloc_validate<<<n, 128, 0, s>>>(base, L, nphase, phase, mat, rve_status);
    NOALLOC_STEP("input validation", cudaGetLastError());
    NOALLOC_STEP("assembly", launch_assemble_fused(tab, ids, n, Fbar, 2, N, 0, s));
    NOALLOC_STEP("factor", launch_factor<float>(tab, ids, n, ws, rve_status, L.kd, L.nr, s));
    NOALLOC_STEP("backward solve", launch_backward<float>(tab, ids, n, ws, 0, L.kd, L.nr, L.nmp, rve_status, s));
    NOALLOC_STEP("residual", launch_residual(tab, ids, n, ws, L.nn, nullptr, s));
    NOALLOC_STEP("Schur complement",
                 launch_schur(tab, ids, n, ws, 1, sigma_eff, Cbar, rve_status, err_est, tol, nullptr, s, 3));
#undef NOALLOC_STEP
    return FE2_OK;
}

extern "C" const char* fe2_noalloc_last_error(void) { return g_err; }
