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
// residual-corrected Schur complement, no refinement sweeps).
#include <cstring>

#include "fe2_internal.cuh"

using namespace fe2;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FE2_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};   // device address of the array, per device

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NoallocLayout {
    int N, nn, nm, kd, nmp, nr;
    size_t off_desc, off_ids, off_tol, off_nbr, off_rve, rve_stride, off_ws, ws_stride, offY, offR, offD, total;
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
        unsigned char* rb = base + L.off_rve + L.rve_stride * t;
        RveDev r{};
        r.N = N;
        r.d = 2;
        r.nm = L.nm;
        r.kd = L.kd;
        r.nn = L.nn;
        r.nphase = nphase;
        r.nm_pad = L.nmp;
        r.nr = L.nr;
        r.phase = phase + (size_t)t * L.nn;
        r.mat = mat + (size_t)t * nphase * 4;
        r.w = nullptr;
        r.stencil = (double*)(rb + L.o_st);
        r.rhs = (double*)(rb + L.o_rhs);
        r.X = (double*)(rb + L.o_X);
        r.KMM = (double*)(rb + L.o_mm);
        r.Pint = r.KMM + 16;
        r.elem = nullptr;
        r.nbr = nbr;
        r.zero_w = 1;
        desc[t] = r;
        ids[t] = t;
    }
    if (t == 0) *(double*)(base + L.off_tol) = tol;
    for (int k = t; k < L.nn * 9; k += gridDim.x * blockDim.x) {
        const int q = k / 9, off = k - 9 * q;
        const int i = unfold_pos(q % N, N), j = unfold_pos(q / N, N);
        const int dx = off % 3 - 1, dy = off / 3 - 1;
        nbr[k] = fold_pos((i + dx + N) % N, N) + N * fold_pos((j + dy + N) % N, N);
    }
}

}  // namespace

extern "C" fe2_status fe2_rve_solve_noalloc(int N, int n, int nphase, const uint8_t* phase, const double* mat,
                                            const double* Fbar, double* sigma_eff, double* Cbar, int* rve_status,
                                            double* err_est, void* cuda_stream) {
    if (N < 3 || n < 1 || nphase < 1 || nphase > MAX_PHASES) return FE2_ERR_ARG;
    if (!phase || !mat || !Fbar || !sigma_eff || !Cbar || !rve_status) return FE2_ERR_ARG;
    const NoallocLayout L = layout_for(N, n);
    if (L.kd + L.nr + 32 > FACT_THREADS) return FE2_ERR_ARG;
    if (L.total > (size_t)FE2_NOALLOC_SCRATCH_BYTES) return FE2_ERR_BUDGET;  // beyond the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FE2_ERR_CUDA;
    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return FE2_ERR_CUDA;
    if ((int)factor_smem_bytes(L.kd, L.nr, false) > smem_optin) return FE2_ERR_ARG;
    // one-time set-up per device (with that device current): the device address
    // of the scratch array; host code must not use the symbol itself
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FE2_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    unsigned char* base = (unsigned char*)g_scratch_addr[dev];
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int setup_threads = 256;
    const int setup_blocks = (n > L.nn * 9 ? n : L.nn * 9) / setup_threads + 1;
    k_noalloc_setup<<<setup_blocks, setup_threads, 0, s>>>(base, L, n, nphase, phase, mat, 1e-10);
    if (cudaGetLastError() != cudaSuccess) return FE2_ERR_CUDA;
    const RveDev* tab = (const RveDev*)(base + L.off_desc);
    const int* ids = (const int*)(base + L.off_ids);
    const double* tol = (const double*)(base + L.off_tol);
    Workspace ws{(char*)base + L.off_ws, L.ws_stride, L.offY, L.offR, L.offD, 0};
    if (launch_check_fbar(Fbar, n, 2, rve_status, s) != cudaSuccess) return FE2_ERR_CUDA;
    if (launch_assemble_fused(tab, ids, n, Fbar, 2, N, 0, s) != cudaSuccess) return FE2_ERR_CUDA;
    if (launch_factor<float>(tab, ids, n, ws, rve_status, L.kd, L.nr, s) != cudaSuccess) return FE2_ERR_CUDA;
    if (launch_backward<float>(tab, ids, n, ws, 0, L.kd, L.nr, L.nmp, rve_status, s) != cudaSuccess)
        return FE2_ERR_CUDA;
    if (launch_residual(tab, ids, n, ws, L.nn, nullptr, s) != cudaSuccess) return FE2_ERR_CUDA;
    if (launch_schur(tab, ids, n, ws, 1, sigma_eff, Cbar, rve_status, err_est, tol, nullptr, s, 3) != cudaSuccess)
        return FE2_ERR_CUDA;
    return FE2_OK;
}
