// bbs_solve_noalloc: the solve for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: hosts whose device memory is already
// reserved by another allocator (a framework's caching pool, a server's
// arena, a fixed budget), and loops that must not wait on the allocator
// (cudaFree synchronises the device, and a cudaMalloc can stall other
// streams). For them the scratch the solve needs (the FP32 copy of the values
// in the mixed-precision mode when they are not staged in shared memory, the
// GMRES basis when it does not fit there) comes from a fixed array compiled
// into the library instead of a caller-provided workspace.
//
// The array is a file-scope static __device__ buffer of kScratchBytes bytes.
// Every GPU that loads the library holds it until the process exits. Host
// code cannot use the array's name as a device address (on the host it names
// a stand-in), so the first call on each device, with that device current,
// looks the address up with cudaGetSymbolAddress and caches it; that first
// call should therefore come before any stream capture. All calls share the
// one array and it keeps the last call's contents: calls that overlap on the
// GPU (different streams, or different host threads) race on it and must be
// serialised by the caller. The solve writes every scratch byte before it
// reads it, so nothing needs clearing between calls.
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/bbs.h"
#include "bbs_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

bbs_status scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices)
        return bbs::record_error(BBS_ERR_UNSUPPORTED, "device index beyond the scratch table");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_ptr[device] == nullptr) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || p == nullptr) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the static scratch: %s",
                     cudaGetErrorString(e));
            return bbs::record_error(BBS_ERR_CUDA, msg);
        }
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return BBS_OK;
}

size_t vals_per_system(const bbs_batch_matrix* A) {
    if (A->fmt == BBS_FMT_CSR) return (size_t)A->nnz;
    if (A->fmt == BBS_FMT_ELL) return (size_t)A->ell_k * (size_t)A->n;
    return (size_t)A->n * (size_t)A->n;
}

}  // namespace

extern "C" bbs_status bbs_solve_noalloc(bbs_handle* handle, const bbs_batch_matrix* A,
                                        const double* b, double* x, const bbs_options* opts,
                                        const bbs_log* log, void* stream) {
    if (handle == nullptr || A == nullptr || opts == nullptr || log == nullptr)
        return bbs::record_error(BBS_ERR_INVALID_ARG, "null handle, matrix, options or log");
    const int device = bbs::handle_device(handle);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return bbs::record_error(BBS_ERR_CUDA, cudaGetErrorString(e));
    size_t need = 0;
    bbs_status s = bbs_workspace_size(handle, A, opts, &need);  // validates A and opts
    if (s != BBS_OK) return s;
    if (A->num_batch == 0) return BBS_OK;
    void* scratch = nullptr;
    if ((s = scratch_address(device, &scratch)) != BBS_OK) return s;
    if (need <= kScratchBytes)
        return bbs_solve(handle, A, b, x, opts, log, scratch, kScratchBytes, stream);

    // Scratch grows linearly with the number of systems, plus parts that do
    // not (the packed-CSR tables, the ILU(0) schedule): size the chunks from
    // the marginal bytes of one more system, then solve them one after the
    // other on the stream.
    bbs_batch_matrix probe = *A;
    size_t one = 0, two = 0;
    probe.num_batch = 1;
    if ((s = bbs_workspace_size(handle, &probe, opts, &one)) != BBS_OK) return s;
    if (one > kScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "one system needs %zu bytes of scratch; the static scratch holds %zu bytes",
                 one, kScratchBytes);
        return bbs::record_error(BBS_ERR_UNSUPPORTED, msg);
    }
    probe.num_batch = 2;
    if ((s = bbs_workspace_size(handle, &probe, opts, &two)) != BBS_OK) return s;
    const size_t per = two > one ? two - one : 1;
    const size_t fixed = one > per ? one - per : 0;
    size_t est = (kScratchBytes - fixed) / per;
    if (est > (size_t)A->num_batch) est = (size_t)A->num_batch;
    int chunk = est < 1 ? 1 : (int)est;
    for (;;) {  // every buffer is rounded up on its own: shrink until it fits
        bbs_batch_matrix c = *A;
        c.num_batch = chunk;
        size_t cneed = 0;
        if ((s = bbs_workspace_size(handle, &c, opts, &cneed)) != BBS_OK) return s;
        if (cneed <= kScratchBytes || chunk == 1) break;
        --chunk;
    }
    const size_t vps = vals_per_system(A), n = (size_t)A->n;
    for (int c0 = 0; c0 < A->num_batch; c0 += chunk) {
        const int cnt = (A->num_batch - c0 < chunk) ? A->num_batch - c0 : chunk;
        bbs_batch_matrix c = *A;
        c.num_batch = cnt;
        c.values = A->values + (size_t)c0 * vps;
        if (A->values_f32 != nullptr) c.values_f32 = A->values_f32 + (size_t)c0 * vps;
        bbs_log lg{log->iters + c0, log->rel_res + c0, log->status + c0,
                   log->inner_iters ? log->inner_iters + c0 : nullptr};
        s = bbs_solve(handle, &c, b + (size_t)c0 * n, x + (size_t)c0 * n, opts, &lg, scratch,
                      kScratchBytes, stream);
        if (s != BBS_OK) return s;
    }
    return BBS_OK;
}
