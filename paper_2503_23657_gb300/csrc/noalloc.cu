// bte_eps_T_noalloc: the convergence measure eps_T of two temperature fields
// with no device allocation at all.
//
// Who needs it: code that cannot call cudaMalloc at the point where it wants
// the measure -- for example a host framework that owns every byte of device
// memory through its own pool, a monitoring loop that must never trigger the
// implicit device synchronisation cudaMalloc may perform, or code running
// while another thread captures a CUDA graph in global mode (where such
// synchronising calls are not allowed).  The regular solver keeps its
// reduction scratch in plan-owned device buffers; this entry point keeps it
// in a fixed file-scope device array instead.
//
// It is a variant of the residual reduction inside the temperature-update
// kernel (update.cu): every block reduces its slice, the last block to
// arrive (ticket counter) combines the block partials in block order, so the
// result is deterministic.  The scratch array is shared by every call on a
// device and keeps the last call's contents; calls that overlap on the GPU
// (different streams without ordering) race on it.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <string>

#include "../../include/bte.h"

namespace bte {
void set_global_error(const std::string &msg);
}

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 1024;
constexpr int kNaMaxDevices = 64;

// [3 * kNaMaxBlocks] block partials {sum of squares, max T, solid count},
// then one 64-bit ticket counter.  24 KB + 8 B per device, held until exit.
static __device__ __align__(256) double g_noalloc_scratch[3 * kNaMaxBlocks + 1];

std::mutex g_na_mutex;
double *g_na_ptr[kNaMaxDevices] = {nullptr};
// id of the context each cached address belongs to: a device reset destroys
// the primary context, the module is loaded again into the next one and the
// array's address may change, so the address is looked up again whenever
// the current context is a different one (context ids are never reused
// within a process)
unsigned long long g_na_ctx[kNaMaxDevices] = {0};

// cuCtxGetCurrent / cuCtxGetId reached through the runtime (no link against
// the driver library)
typedef CUresult (*NaCtxGetCurrent)(CUcontext *);
typedef CUresult (*NaCtxGetId)(CUcontext, unsigned long long *);

bool na_current_context_id(unsigned long long *id) {
    static NaCtxGetCurrent get_current = nullptr;
    static NaCtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return false;
        }
        get_current = reinterpret_cast<NaCtxGetCurrent>(f1);
        get_id = reinterpret_cast<NaCtxGetId>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

__device__ __forceinline__ void na_block_reduce(double &a, double &m, double &n, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        n += __shfl_down_sync(0xffffffffu, n, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[3 * warp] = a;
        sh[3 * warp + 1] = m;
        sh[3 * warp + 2] = n;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? sh[3 * lane] : 0.0;
        m = lane < nw ? sh[3 * lane + 1] : -INFINITY;
        n = lane < nw ? sh[3 * lane + 2] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
            n += __shfl_down_sync(0xffffffffu, n, o);
        }
    }
}

__global__ void __launch_bounds__(kNaThreads)
eps_noalloc_kernel(const double *__restrict__ T_old, const double *__restrict__ T_new,
                   const uint8_t *__restrict__ mask, long long N, double *scratch, double *out) {
    __shared__ double sh[3 * (kNaThreads / 32)];
    __shared__ int is_last;
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(scratch + 3 * kNaMaxBlocks);
    double ss = 0.0, mx = -INFINITY, cnt = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += stride) {
        if (mask != nullptr && mask[c] == 0) continue;
        const double tn = T_new[c];
        const double d = T_old[c] - tn;
        ss += d * d;
        mx = fmax(mx, tn);
        cnt += 1.0;
    }
    na_block_reduce(ss, mx, cnt, sh);
    if (threadIdx.x == 0) {
        scratch[3 * blockIdx.x] = ss;
        scratch[3 * blockIdx.x + 1] = mx;
        scratch[3 * blockIdx.x + 2] = cnt;
        __threadfence();
        is_last = (atomicAdd(counter, 1ull) == (unsigned long long)(gridDim.x - 1));
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double tss = 0.0, tmx = -INFINITY, tn = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        tss += __ldcg(&scratch[3 * i]);
        tmx = fmax(tmx, __ldcg(&scratch[3 * i + 1]));
        tn += __ldcg(&scratch[3 * i + 2]);
    }
    na_block_reduce(tss, tmx, tn, sh);
    if (threadIdx.x == 0) {
        // NaN anywhere: NaN (fmax skips NaN, so the maximum alone cannot tell)
        out[0] = isnan(tss) || isnan(tmx) ? NAN : ((tn > 0.0 && tmx > 0.0) ? sqrt(tss / tn) / tmx : 0.0);
        out[1] = tmx;
        out[2] = tn;
        *counter = 0ull;  // ready for the next call
    }
}

int na_fail(int code, const char *msg) {
    bte::set_global_error(msg);
    return code;
}

}  // namespace

extern "C" int bte_eps_T_noalloc(const double *T_old, const double *T_new, const uint8_t *mask, long long N,
                                 double *out, void *stream) {
    if (!T_old || !T_new || !out) return na_fail(BTE_EINVAL, "bte_eps_T_noalloc: null pointer");
    if (N < 1 || N > BTE_NOALLOC_MAX_CELLS)
        return na_fail(BTE_EINVAL, "bte_eps_T_noalloc: N must be in [1, BTE_NOALLOC_MAX_CELLS]");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
        cudaGetLastError();
        return na_fail(BTE_ECUDA, "bte_eps_T_noalloc: no usable current CUDA device");
    }
    // (before the runtime has made its context on this device there is no
    // current context yet; the symbol lookup below makes it)
    unsigned long long ctx_id = 0;
    const bool have_ctx = na_current_context_id(&ctx_id);
    double *scratch = nullptr;
    {
        // once per device and context, with that device current: the device
        // address of the file-scope scratch array (its host-side name is not
        // a device address and must never be passed to a kernel)
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!have_ctx || g_na_ptr[dev] == nullptr || g_na_ctx[dev] != ctx_id) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || p == nullptr || !na_current_context_id(&ctx_id)) {
                cudaGetLastError();
                g_na_ptr[dev] = nullptr;
                return na_fail(BTE_ECUDA, "bte_eps_T_noalloc: cudaGetSymbolAddress failed");
            }
            g_na_ptr[dev] = static_cast<double *>(p);
            g_na_ctx[dev] = ctx_id;
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the ticket counter must start at zero
    cudaError_t e = cudaMemsetAsync(scratch + 3 * kNaMaxBlocks, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return na_fail(BTE_ECUDA, "bte_eps_T_noalloc: cudaMemsetAsync failed");
    const long long want = (N + kNaThreads - 1) / kNaThreads;
    const int blocks = (int)(want < kNaMaxBlocks ? want : kNaMaxBlocks);
    eps_noalloc_kernel<<<blocks, kNaThreads, 0, st>>>(T_old, T_new, mask, N, scratch, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(BTE_ECUDA, "bte_eps_T_noalloc: launch failed");
    return BTE_OK;
}
