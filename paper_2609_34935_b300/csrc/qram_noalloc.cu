// qram_noalloc.cu -- the allocation-free entry point qram_run_static.
//
// Some callers must not allocate device memory while they run: a host with
// a fixed device-memory plan decided at start-up (real-time or embedded
// deployments), code that runs inside another framework's allocator and may
// not go around it, or a process that has already handed all device memory
// to a pool.  qram_run_static serves them: the caller passes every input and
// output as device pointers, and the per-CTA scratch of the trajectory
// kernel comes from one file-scope device array of fixed size instead of
// cudaMalloc.  This file calls no cudaMalloc, cudaFree or other allocating
// routine.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda.h>            // driver types only: the two driver calls are looked up at run time
#include <cuda_runtime.h>

#include "qram_internal.h"

using namespace qram;

namespace {
// Bytes of the shared static scratch.  The first 256 bytes hold the work
// counter and the input-validation flag; the rest is per-CTA scratch.
constexpr size_t kStaticBytes = size_t(32) << 20;
constexpr size_t kHeader = 256;
constexpr int kMaxDevices = 64;
}  // namespace

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_qram_static_scratch[kStaticBytes];

namespace {

std::mutex g_mu;
// Per device: the context the array's address was looked up in, and that
// address.  A device reset (or any teardown of the context) reloads the
// module at a new address, so the cached one is only valid in its context.
unsigned long long g_ctx[kMaxDevices] = {};
void *g_base[kMaxDevices] = {};

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// Unique id of the context current on this thread (0 on failure).  The
// driver calls come through the runtime's entry-point query, so the library
// does not link the driver library itself.
unsigned long long current_ctx_id() {
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return 0;
        }
        get_current = (PfnCtxGetCurrent)f1;
        get_id = (PfnCtxGetId)f2;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Once per device and context, with that device current: the device address
// of the static array (the host-side symbol is only a stand-in, not an
// address).  Looked up again when the current context is not the one of the
// cached address (after a device reset, or under another context).
int static_setup(int device, size_t dyn, void **base, int *resident_slots) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (device < 0 || device >= kMaxDevices) return QRAM_E_ARG;
    unsigned long long ctx = current_ctx_id();
    if (ctx == 0) {
        // no context current yet: make the device's primary context current
        // (this initialises it); a context the caller made current is kept
        if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return QRAM_E_CUDA; }
        ctx = current_ctx_id();
        if (ctx == 0) return QRAM_E_CUDA;
    }
    if (!g_base[device] || g_ctx[device] != ctx) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_qram_static_scratch);
        if (e != cudaSuccess || !p) { cudaGetLastError(); return QRAM_E_CUDA; }
        g_base[device] = p;
        g_ctx[device] = ctx;
    }
    *base = g_base[device];
    *resident_slots = resident_slots_per_device(device, kernel_threads(), dyn);
    if (*resident_slots < 1) return QRAM_E_CUDA;
    return QRAM_OK;
}

// One CTA checks the device-resident problem: addresses distinct and below
// 2^n, bus words and memory cells below 2^k, sum |amp|^2 = 1 within 1e-12.
__global__ void __launch_bounds__(1024) validate_kernel(const uint8_t *mem, const uint32_t *addr, const uint32_t *bus,
                                                        const double *re, const double *im, int n, int k, int D,
                                                        uint32_t *err) {
    __shared__ uint32_t seen[512];
    __shared__ double part[32];
    for (int w = threadIdx.x; w < 512; w += blockDim.x) seen[w] = 0;
    __syncthreads();
    bool bad = false;
    const uint32_t N = 1u << n, K = 1u << k;
    for (uint32_t c = threadIdx.x; c < N; c += blockDim.x) if (mem[c] >= K) bad = true;
    double s = 0.0;
    for (int b = threadIdx.x; b < D; b += blockDim.x) {
        const uint32_t a = addr[b];
        if (a >= N || bus[b] >= K) { bad = true; continue; }
        const uint32_t old = atomicOr(&seen[a >> 5], 1u << (a & 31u));
        if (old & (1u << (a & 31u))) bad = true;
        s += re[b] * re[b] + im[b] * im[b];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (bad) atomicOr(err, 1u);
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        if (!(t > 1.0 - 1e-12 && t < 1.0 + 1e-12)) atomicOr(err, 1u);
    }
}

}  // namespace

extern "C" int qram_run_static(int mode, int32_t encoding, int32_t n, int32_t k, int32_t num_branches,
                               const uint8_t *memory, const uint32_t *addr, const uint32_t *bus,
                               const double *amp_re, const double *amp_im, uint64_t seed, uint64_t traj0,
                               uint32_t ntraj, const double *gamma, double gamma_max, qram_result_t *out,
                               void *cuda_stream) {
    if (mode != 0 && mode != 1) return QRAM_E_ARG;
    if (encoding != QRAM_QUTRIT && encoding != QRAM_QUBIT) return QRAM_E_ARG;
    if (n < 1 || n > kMaxN || k < 1 || k > kMaxK || k > n) return QRAM_E_ARG;
    if (num_branches < 1 || num_branches > (1 << n)) return QRAM_E_ARG;
    if (!memory || !addr || !bus || !amp_re || !amp_im || !gamma || !out) return QRAM_E_ARG;
    if (!(gamma_max >= 0.0 && gamma_max < gamma_limit(n, k))) return QRAM_E_ARG;
    if (ntraj == 0) return QRAM_OK;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return QRAM_E_CUDA;
    void *base = nullptr;
    int resident = 0;
    const size_t dyn = dyn_smem_bytes(n, k);
    int rc = static_setup(device, dyn, &base, &resident);
    if (rc) return rc;
    // as many CTA slots as fit in the static array (at most one per resident CTA)
    const size_t avail = kStaticBytes - kHeader;
    const int threads = kernel_threads();
    const size_t one = carve_scratch(encoding, n, k, num_branches, 1, gamma_max, threads, nullptr, nullptr);
    if (one > avail) return QRAM_E_TOOBIG;
    int slots = (int)std::min<size_t>((size_t)resident, avail / one);
    while (slots > 1 && carve_scratch(encoding, n, k, num_branches, slots, gamma_max, threads, nullptr, nullptr) > avail) --slots;
    Params P;
    std::memset(&P, 0, sizeof(P));
    if (build_ops(n, k, P.ops) != QRAM_OK) return QRAM_E_ARG;
    build_occupancy(n, k, P.ops, P.occ2);
    build_orbit(n, k, P.ops, &P.orbit);
    P.enc = encoding; P.n = n; P.k = k; P.T = 6 * n + 2 * k; P.D = num_branches;
    P.nodes = (1 << n) - 1; P.M = 2 * P.nodes; P.nthreads = threads; P.hist_pad = hist_pad(n, k);
    P.gamma_lim = gamma_limit(n, k);
    P.mem = memory; P.addr = addr; P.bus = bus; P.amp_re = amp_re; P.amp_im = amp_im;
    P.seed = seed; P.traj0 = traj0; P.ntraj = ntraj; P.gamma = gamma;
    P.mode = mode == 0 ? kPruned : kFull;
    P.out = out;
    char *b = (char *)base;
    P.work = (uint32_t *)b;
    P.input_error = (const uint32_t *)(b + 4);
    P.w2u = (const double *)(b + 8);
    carve_scratch(encoding, n, k, num_branches, slots, gamma_max, threads, b + kHeader, &P.scr);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the array keeps the previous call's contents: reset the counter and the flag
    if (cudaMemsetAsync(b, 0, kHeader, st) != cudaSuccess) return QRAM_E_CUDA;
    validate_kernel<<<1, 1024, 0, st>>>(memory, addr, bus, amp_re, amp_im, n, k, num_branches, (uint32_t *)(b + 4));
    if (cudaGetLastError() != cudaSuccess) return QRAM_E_CUDA;
    if (launch_uniform_weight(amp_re, amp_im, num_branches, encoding == QRAM_QUBIT ? k : 0, (double *)(b + 8), st) != cudaSuccess)
        return QRAM_E_CUDA;
    const int grid = (int)std::min<uint32_t>((uint32_t)slots, ntraj);
    if (launch_trajectories(P, grid, threads, dyn, st) != cudaSuccess) return QRAM_E_CUDA;
    return QRAM_OK;
}
