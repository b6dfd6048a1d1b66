// Uneven batches, host side: plan, autotuner and CUDA-graph capture of the
// persistent launch (kernel in bbs_varsize.cuh).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bbs.h"
#include "bbs_internal.h"
#include "bbs_varsize.cuh"

// ------------------------------------------------------------------ host

struct bbs_var_plan {
    int device = 0;
    int num_batch = 0;
    int rmax = 8, threads = 256, grid = 0;
    size_t smem = 0;
    const void* fn = nullptr;
    bbs::VarParams P{};
    int32_t* d_order = nullptr;
    int32_t* d_counters = nullptr;
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t knode = nullptr;
};

namespace {

using bbs::record_error;

bbs_status errf(bbs_status s, const char* fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    return record_error(s, msg);
}

bbs_status cuda_err(cudaError_t e, const char* what) {
    return errf(BBS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

const int kEdges[] = {32, 64, 128, 256, 512, 1024, 2048};

bbs_status check_batch(const bbs_var_batch* vb, const bbs_var_host_info* host, const bbs_options* o) {
    if (vb == nullptr || host == nullptr || o == nullptr)
        return errf(BBS_ERR_INVALID_ARG, "null batch, host info or options");
    if (vb->num_batch < 0 || vb->num_patterns < 1)
        return errf(BBS_ERR_INVALID_ARG, "need num_batch >= 0 and num_patterns >= 1");
    if (!vb->pat_n || !vb->pat_nnz || !vb->pat_rp_off || !vb->pat_ci_off || !vb->row_ptrs ||
        !vb->col_idxs || !vb->sys_pattern || !vb->val_off || !vb->vec_off || !vb->values)
        return errf(BBS_ERR_INVALID_ARG, "a device array of the batch is NULL");
    if (!host->pat_n || !host->pat_nnz || !host->sys_pattern)
        return errf(BBS_ERR_INVALID_ARG, "a host metadata array is NULL");
    if (o->solver != BBS_SOLVER_BICGSTAB && o->solver != BBS_SOLVER_CG)
        return errf(BBS_ERR_UNSUPPORTED, "uneven batches run BiCGSTAB or CG");
    if (o->precision != BBS_PRECISION_FP64)
        return errf(BBS_ERR_UNSUPPORTED, "uneven batches run in FP64");
    if (o->precond < 0 || o->precond > 1 || o->tol_type < 0 || o->tol_type > 1 || !(o->tol > 0.0) ||
        o->max_iters < 0)
        return errf(BBS_ERR_INVALID_ARG, "invalid preconditioner, tolerance or iteration cap");
    for (int p = 0; p < vb->num_patterns; ++p)
        if (host->pat_n[p] <= 0 || host->pat_n[p] > 2048 || host->pat_nnz[p] < 0)
            return errf(BBS_ERR_INVALID_ARG, "pattern %d: n must be in [1, 2048], nnz >= 0", p);
    for (int i = 0; i < vb->num_batch; ++i)
        if (host->sys_pattern[i] < 0 || host->sys_pattern[i] >= vb->num_patterns)
            return errf(BBS_ERR_INVALID_ARG, "system %d names pattern %d of %d", i, host->sys_pattern[i],
                        vb->num_patterns);
    return BBS_OK;
}

bbs_status check_tuning(const bbs_var_tuning* t) {
    if (t->num_buckets < 1 || t->num_buckets > 8) return errf(BBS_ERR_INVALID_ARG, "num_buckets must be 1..8");
    if (t->block_warps != 8 && t->block_warps != 16) return errf(BBS_ERR_INVALID_ARG, "block_warps must be 8 or 16");
    for (int b = 0; b < t->num_buckets; ++b) {
        if (b > 0 && t->bucket_max_n[b] <= t->bucket_max_n[b - 1])
            return errf(BBS_ERR_INVALID_ARG, "bucket_max_n must be ascending");
        if (!is_pow2(t->team_warps[b]) || t->team_warps[b] > 16)
            return errf(BBS_ERR_INVALID_ARG, "team_warps must be 1, 2, 4, 8 or 16");
        if (t->stage_values[b] != 0 && t->stage_values[b] != 1)
            return errf(BBS_ERR_INVALID_ARG, "stage_values must be 0 or 1");
    }
    return BBS_OK;
}

struct PlanInputs {
    const bbs_var_batch* vb;
    const bbs_var_host_info* host;
    const bbs_options* o;
    bbs_var_tuning t;
    const int* subset;  // systems to schedule (null = all)
    int nsubset;
};

bbs_status build_plan(bbs_handle* h, const PlanInputs& in, bbs_var_plan** out) {
    const bbs_var_batch* vb = in.vb;
    const bbs_var_tuning& t = in.t;
    const int rmax = t.block_warps == 8 ? 8 : 4;
    const int nb = in.subset ? in.nsubset : vb->num_batch;
    std::vector<int> sys(nb);
    for (int i = 0; i < nb; ++i) sys[i] = in.subset ? in.subset[i] : i;

    // team warps per bucket: at least what the rows need, never more than a larger bucket's
    const int B = t.num_buckets;
    std::vector<int> nmax(B, 0), W(B), bucket(nb);
    for (int i = 0; i < nb; ++i) {
        const int n = in.host->pat_n[in.host->sys_pattern[sys[i]]];
        int b = 0;
        while (b < B && n > t.bucket_max_n[b]) ++b;
        if (b == B) return errf(BBS_ERR_INVALID_ARG, "system %d (n = %d) exceeds the last bucket", sys[i], n);
        bucket[i] = b;
        nmax[b] = std::max(nmax[b], n);
    }
    for (int b = 0; b < B; ++b) {
        const int need = pow2_at_least((std::max(nmax[b], 1) + 32 * rmax - 1) / (32 * rmax));
        W[b] = std::max(t.team_warps[b], need);
    }
    for (int b = B - 2; b >= 0; --b) W[b] = std::min(W[b], W[b + 1]);
    for (int b = 0; b < B; ++b)
        if (W[b] > t.block_warps)
            return errf(BBS_ERR_UNSUPPORTED, "bucket %d needs %d warps per system, the block has %d", b, W[b],
                        t.block_warps);

    // order: team size descending, staging, then estimated cost descending
    std::vector<double> cost(nb);
    for (int i = 0; i < nb; ++i) {
        const int p = in.host->sys_pattern[sys[i]];
        const double n = in.host->pat_n[p], nz = in.host->pat_nnz[p];
        cost[i] = (2.0 * nz + 14.0 * n) * std::sqrt(n);
    }
    std::vector<int> idx(nb);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) {
        const int wa = W[bucket[a]], wc = W[bucket[c]];
        if (wa != wc) return wa > wc;
        const int sa = t.stage_values[bucket[a]], sc = t.stage_values[bucket[c]];
        if (sa != sc) return sa > sc;
        return cost[a] > cost[c];
    });

    bbs_var_plan* pl = new bbs_var_plan();
    bbs::VarParams& P = pl->P;
    P.num_segments = 0;
    std::vector<int32_t> order(nb);
    std::vector<int> seg_nmax, seg_nnzmax;
    for (int k = 0; k < nb; ++k) {
        const int i = idx[k];
        order[k] = sys[i];
        const int w = W[bucket[i]], st = t.stage_values[bucket[i]];
        const int p = in.host->sys_pattern[sys[i]];
        if (P.num_segments == 0 || P.seg_warps[P.num_segments - 1] != w ||
            P.seg_stage[P.num_segments - 1] != st) {
            if (P.num_segments == bbs::kMaxSeg) {
                delete pl;
                return errf(BBS_ERR_UNSUPPORTED, "more than %d segments", bbs::kMaxSeg);
            }
            P.seg_begin[P.num_segments] = k;
            P.seg_count[P.num_segments] = 0;
            P.seg_warps[P.num_segments] = w;
            P.seg_stage[P.num_segments] = st;
            seg_nmax.push_back(0);
            seg_nnzmax.push_back(0);
            ++P.num_segments;
        }
        const int s = P.num_segments - 1;
        ++P.seg_count[s];
        seg_nmax[s] = std::max(seg_nmax[s], in.host->pat_n[p]);
        seg_nnzmax[s] = std::max(seg_nnzmax[s], in.host->pat_nnz[p]);
    }
    // per-warp shared-memory slice: a team of w warps uses w consecutive slices
    size_t slice = 16;
    for (int s = 0; s < P.num_segments; ++s) {
        const size_t npad = (size_t)((seg_nmax[s] + 1) & ~1);
        size_t need = 16 + (256 + 2 * npad) * 8;
        if (P.seg_stage[s]) need += ((size_t)seg_nnzmax[s] * 8 + 15) / 16 * 16;
        const size_t per = (need + P.seg_warps[s] - 1) / P.seg_warps[s];
        slice = std::max(slice, (per + 15) / 16 * 16);
    }
    pl->rmax = rmax;
    pl->threads = 32 * t.block_warps;
    pl->smem = slice * (size_t)t.block_warps;
    P.slice_bytes = (int)slice;
    int dev = bbs::handle_device(h), sms = 0, optin = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (pl->smem > (size_t)optin) {
        delete pl;
        return errf(BBS_ERR_UNSUPPORTED, "the plan needs %zu bytes of shared memory per block (max %d)",
                    pl->smem, optin);
    }
    pl->device = dev;
    pl->num_batch = nb;
    pl->fn = rmax == 8 ? bbs::varsize_kernel8_fn() : bbs::varsize_kernel4_fn();
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(pl->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl->smem)) !=
        cudaSuccess) {
        delete pl;
        return cuda_err(e, "cudaFuncSetAttribute");
    }
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl->fn, pl->threads, pl->smem)) !=
            cudaSuccess ||
        per_sm < 1) {
        delete pl;
        return e != cudaSuccess ? cuda_err(e, "occupancy query")
                                : errf(BBS_ERR_UNSUPPORTED, "the persistent block does not fit on an SM");
    }
    pl->grid = per_sm * sms;

    P.pat_n = vb->pat_n;
    P.pat_nnz = vb->pat_nnz;
    P.rp_off = vb->pat_rp_off;
    P.ci_off = vb->pat_ci_off;
    P.row_ptrs = vb->row_ptrs;
    P.col_idxs = vb->col_idxs;
    P.sys_pattern = vb->sys_pattern;
    P.val_off = vb->val_off;
    P.vec_off = vb->vec_off;
    P.values = vb->values;
    P.solver = in.o->solver;
    P.cfg.precond = in.o->precond;
    P.cfg.tol_type = in.o->tol_type;
    P.cfg.max_iters = in.o->max_iters;
    P.cfg.restart = 0;
    P.cfg.max_outer = 0;
    P.cfg.tol = in.o->tol;
    P.cfg.inner_tol = 0.0;
    P.cfg.ws = nullptr;

    if ((e = cudaMalloc(&pl->d_order, sizeof(int32_t) * std::max(nb, 1))) != cudaSuccess ||
        (e = cudaMalloc(&pl->d_counters, sizeof(int32_t) * bbs::kMaxSeg)) != cudaSuccess) {
        bbs_var_plan_destroy(pl);
        return errf(BBS_ERR_NO_MEMORY, "plan buffers: %s", cudaGetErrorString(e));
    }
    if (nb > 0 && (e = cudaMemcpy(pl->d_order, order.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice)) !=
                      cudaSuccess) {
        bbs_var_plan_destroy(pl);
        return cuda_err(e, "order upload");
    }
    P.order = pl->d_order;
    P.counters = pl->d_counters;

    // graph: reset the counters, then the persistent launch
    if ((e = cudaStreamCreateWithFlags(&pl->capture, cudaStreamNonBlocking)) != cudaSuccess) {
        bbs_var_plan_destroy(pl);
        return cuda_err(e, "capture stream");
    }
    e = cudaStreamBeginCapture(pl->capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(pl->d_counters, 0, sizeof(int32_t) * bbs::kMaxSeg, pl->capture);
        void* args[] = {&P};
        cudaLaunchKernel(pl->fn, dim3(pl->grid), dim3(pl->threads), args, pl->smem, pl->capture);
        e = cudaStreamEndCapture(pl->capture, &pl->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
    if (e == cudaSuccess) {
        size_t count = 0;
        cudaGraphGetNodes(pl->graph, nullptr, &count);
        std::vector<cudaGraphNode_t> nodes(count);
        cudaGraphGetNodes(pl->graph, nodes.data(), &count);
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) pl->knode = nd;
        }
        if (pl->knode == nullptr) e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) {
        bbs_var_plan_destroy(pl);
        return cuda_err(e, "graph capture");
    }
    *out = pl;
    return BBS_OK;
}

void default_tuning(int32_t max_n, bbs_var_tuning* t) {
    std::memset(t, 0, sizeof *t);
    t->block_warps = 8;
    int b = 0;
    for (int e : kEdges) {
        t->bucket_max_n[b] = e;
        t->team_warps[b] = pow2_at_least((e + 32 * 5 - 1) / (32 * 5));
        t->stage_values[b] = 0;
        ++b;
        if (e >= max_n) break;
    }
    t->num_buckets = b;
}

}  // namespace

extern "C" {

bbs_status bbs_var_default_tuning(int32_t max_n, bbs_var_tuning* tuning) {
    if (tuning == nullptr || max_n < 1 || max_n > 2048)
        return errf(BBS_ERR_INVALID_ARG, "need a tuning pointer and 1 <= max_n <= 2048");
    default_tuning(max_n, tuning);
    return BBS_OK;
}

bbs_status bbs_var_plan_create(bbs_handle* h, const bbs_var_batch* vb, const bbs_var_host_info* host,
                               const bbs_options* o, const bbs_var_tuning* tuning, bbs_var_plan** plan) {
    if (h == nullptr || plan == nullptr) return errf(BBS_ERR_INVALID_ARG, "null handle or plan pointer");
    *plan = nullptr;
    bbs_status s = check_batch(vb, host, o);
    if (s != BBS_OK) return s;
    PlanInputs in{vb, host, o, {}, nullptr, 0};
    if (tuning) {
        in.t = *tuning;
    } else {
        int mx = 1;
        for (int p = 0; p < vb->num_patterns; ++p) mx = std::max(mx, host->pat_n[p]);
        default_tuning(mx, &in.t);
    }
    if ((s = check_tuning(&in.t)) != BBS_OK) return s;
    cudaSetDevice(bbs::handle_device(h));
    return build_plan(h, in, plan);
}

bbs_status bbs_var_solve(bbs_var_plan* pl, const double* b, double* x, const bbs_log* log, void* stream) {
    if (pl == nullptr || log == nullptr || !log->iters || !log->rel_res || !log->status)
        return errf(BBS_ERR_INVALID_ARG, "null plan or log arrays");
    if (pl->num_batch > 0 && (b == nullptr || x == nullptr)) return errf(BBS_ERR_INVALID_ARG, "null b or x");
    cudaSetDevice(pl->device);
    pl->P.b = b;
    pl->P.x = x;
    pl->P.iters = log->iters;
    pl->P.rel_res = log->rel_res;
    pl->P.status = log->status;
    void* args[] = {&pl->P};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(pl->fn);
    kp.gridDim = dim3(pl->grid);
    kp.blockDim = dim3(pl->threads);
    kp.sharedMemBytes = (unsigned)pl->smem;
    kp.kernelParams = args;
    cudaError_t e = cudaGraphExecKernelNodeSetParams(pl->exec, pl->knode, &kp);
    if (e != cudaSuccess) return cuda_err(e, "graph parameter update");
    if ((e = cudaGraphLaunch(pl->exec, reinterpret_cast<cudaStream_t>(stream))) != cudaSuccess)
        return cuda_err(e, "graph launch");
    return BBS_OK;
}

bbs_status bbs_var_plan_destroy(bbs_var_plan* pl) {
    if (pl == nullptr) return BBS_OK;
    cudaSetDevice(pl->device);
    cudaDeviceSynchronize();
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->capture) cudaStreamDestroy(pl->capture);
    if (pl->d_order) cudaFree(pl->d_order);
    if (pl->d_counters) cudaFree(pl->d_counters);
    delete pl;
    return BBS_OK;
}

bbs_status bbs_var_tune(bbs_handle* h, const bbs_var_batch* vb, const bbs_var_host_info* host,
                        const double* b, const double* x0, const bbs_options* o, int32_t sample,
                        bbs_var_tuning* tuning) {
    if (h == nullptr || tuning == nullptr || b == nullptr || x0 == nullptr || sample < 1)
        return errf(BBS_ERR_INVALID_ARG, "null argument or sample < 1");
    bbs_status s = check_batch(vb, host, o);
    if (s != BBS_OK) return s;
    cudaSetDevice(bbs::handle_device(h));
    int mx = 1;
    for (int p = 0; p < vb->num_patterns; ++p) mx = std::max(mx, host->pat_n[p]);
    bbs_var_tuning base;
    default_tuning(mx, &base);
    const int B = base.num_buckets;
    // members of each bucket, sampled evenly
    std::vector<std::vector<int>> members(B);
    for (int i = 0; i < vb->num_batch; ++i) {
        const int n = host->pat_n[host->sys_pattern[i]];
        int k = 0;
        while (k < B - 1 && n > base.bucket_max_n[k]) ++k;
        members[k].push_back(i);
    }
    // Each trial must fill the GPU several times over, or it measures the
    // latency of one system instead of the throughput of many: at least
    // 4 x (SMs x 16 warps) systems per bucket when the bucket has them.
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, bbs::handle_device(h));
    const size_t want = std::max<size_t>((size_t)sample, (size_t)sms * 16 * 4);
    std::vector<std::vector<int>> samp(B);
    for (int k = 0; k < B; ++k) {
        const size_t m = members[k].size();
        const size_t c = std::min<size_t>(m, want);
        for (size_t j = 0; j < c; ++j) samp[k].push_back(members[k][j * m / c]);
    }
    // private scratch: x and the log, covering the batch's index ranges
    int64_t vec_len = 0;
    {
        std::vector<int64_t> vo(vb->num_batch);
        if (vb->num_batch > 0)
            cudaMemcpy(vo.data(), vb->vec_off, sizeof(int64_t) * vb->num_batch, cudaMemcpyDeviceToHost);
        for (int i = 0; i < vb->num_batch; ++i)
            vec_len = std::max<int64_t>(vec_len, vo[i] + host->pat_n[host->sys_pattern[i]]);
    }
    double *dx = nullptr, *drr = nullptr;
    int32_t *dit = nullptr, *dst = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&dx, sizeof(double) * std::max<int64_t>(vec_len, 1))) != cudaSuccess ||
        (e = cudaMalloc(&drr, sizeof(double) * std::max(vb->num_batch, 1))) != cudaSuccess ||
        (e = cudaMalloc(&dit, sizeof(int32_t) * std::max(vb->num_batch, 1))) != cudaSuccess ||
        (e = cudaMalloc(&dst, sizeof(int32_t) * std::max(vb->num_batch, 1))) != cudaSuccess) {
        cudaFree(dx); cudaFree(drr); cudaFree(dit); cudaFree(dst);
        return errf(BBS_ERR_NO_MEMORY, "tuner scratch: %s", cudaGetErrorString(e));
    }
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    bbs_log lg{dit, drr, dst, nullptr};

    bbs_var_tuning best_overall = base;
    double best_total = INFINITY;
    for (int bw : {8, 16}) {
        bbs_var_tuning cand = base;
        cand.block_warps = bw;
        const int rmax = bw == 8 ? 8 : 4;
        double total = 0.0;
        bool feasible = true;
        for (int k = 0; k < B && feasible; ++k) {
            if (samp[k].empty()) continue;
            int nk = 0;
            for (int i : samp[k]) nk = std::max(nk, host->pat_n[host->sys_pattern[i]]);
            const int wmin = pow2_at_least((nk + 32 * rmax - 1) / (32 * rmax));
            double best = INFINITY;
            int bestw = wmin, bests = 0;
            for (int w = wmin; w <= bw; w *= 2) {
                for (int stg = 0; stg <= 1; ++stg) {
                    PlanInputs in{vb, host, o, {}, samp[k].data(), (int)samp[k].size()};
                    std::memset(&in.t, 0, sizeof in.t);
                    in.t.num_buckets = 1;
                    in.t.bucket_max_n[0] = 2048;
                    in.t.team_warps[0] = w;
                    in.t.stage_values[0] = stg;
                    in.t.block_warps = bw;
                    bbs_var_plan* pl = nullptr;
                    if (build_plan(h, in, &pl) != BBS_OK) continue;
                    float ms_sum = 0.f;
                    bool ok = true;
                    for (int rep = 0; rep < 3 && ok; ++rep) {
                        cudaMemcpyAsync(dx, x0, sizeof(double) * vec_len, cudaMemcpyDeviceToDevice, st);
                        cudaEventRecord(e0, st);
                        ok = bbs_var_solve(pl, b, dx, &lg, st) == BBS_OK;
                        cudaEventRecord(e1, st);
                        cudaEventSynchronize(e1);
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (rep > 0) ms_sum += ms;
                    }
                    bbs_var_plan_destroy(pl);
                    if (!ok) continue;
                    const double per = ms_sum / 2.0 / samp[k].size();
                    if (per < best) {
                        best = per;
                        bestw = w;
                        bests = stg;
                    }
                }
            }
            if (!std::isfinite(best)) {
                feasible = false;
                break;
            }
            cand.team_warps[k] = bestw;
            cand.stage_values[k] = bests;
            total += best * members[k].size();
        }
        if (feasible && total < best_total) {
            best_total = total;
            best_overall = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(dx);
    cudaFree(drr);
    cudaFree(dit);
    cudaFree(dst);
    if (!std::isfinite(best_total)) return errf(BBS_ERR_UNSUPPORTED, "no feasible launch choice");
    *tuning = best_overall;
    return BBS_OK;
}

}  // extern "C"
