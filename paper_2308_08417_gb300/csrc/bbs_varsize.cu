// Uneven batches, host side: plan, autotuner and the CUDA graph of the
// persistent team launch (kernel in bbs_varsize.cuh) and of the packed
// small-system launches (bbs_varpacked.cuh).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bbs.h"
#include "bbs_internal.h"
#include "bbs_kernels.h"
#include "bbs_varpacked.cuh"
#include "bbs_varwide.cuh"
#include "bbs_varsize.cuh"

namespace bbs {
const void* varpacked_fn(int solver, int L, int R) {
    return L == 4 ? varpacked_fn_l4(solver, R) : L == 8 ? varpacked_fn_l8(solver, R) : varpacked_fn_l16(solver, R);
}
const void* varwide_fn(int R) { return R <= 12 ? varwide_fn_lo(R) : varwide_fn_hi(R); }
}  // namespace bbs

// ------------------------------------------------------------------ host

struct PackedClass {
    int L = 0, R = 0, grid = 0;
    size_t smem = 0;
    const void* fn = nullptr;
    bbs::VarPackedParams P{};
    cudaGraphNode_t node = nullptr;
};

struct WideClass {
    int warps = 0, R = 0;
    size_t smem = 0;
    const void* fn = nullptr;
    bbs::VarWideParams P{};
    cudaGraphNode_t node = nullptr;
};

struct bbs_var_plan {
    int device = 0;
    int num_batch = 0;
    int rmax = 8, threads = 256, grid = 0;
    size_t smem = 0;
    const void* fn = nullptr;
    bbs::VarParams P{};
    int team_count = 0;  // systems of the persistent launch
    bool has_team = false;
    int packed_count = 0;
    std::vector<PackedClass> classes;
    int wide_count = 0;
    std::vector<WideClass> wides;
    int32_t* d_order = nullptr;
    int32_t* d_counters = nullptr;
    int32_t* d_tables = nullptr;  // flag [4] | xcols | xsrc of the packed patterns
    int64_t* d_tab_off = nullptr;
    int32_t* d_tab_k = nullptr;
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
        if (t->pack[b] != 0 && t->pack[b] != 1) return errf(BBS_ERR_INVALID_ARG, "pack must be 0 or 1");
        if (t->wide[b] < 0 || t->wide[b] > 3) return errf(BBS_ERR_INVALID_ARG, "wide must be 0..3");
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

// Packed small systems (bbs_varpacked.cuh): a class (L, R) per pattern,
// chosen by the rule of the uniform packed kernels: the narrowest group of 4,
// 8 or 16 lanes that covers n in at most kMaxPackedR rows per lane and leaves
// at least kVarPackedMinWarps one-warp blocks resident per SM.
constexpr int kVarPackMaxN = 16 * bbs::kMaxPackedR;
constexpr int kVarPackedMinWarps = 8;

struct PatPack {
    int state = 0;  // 0 not examined, 1 packed, 2 left to the teams
    int L = 0, R = 0, k = 0;
    size_t raw = 0;  // shared-memory bytes of one group before the bank shift
};

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// A group's bytes padded to 8 L past a multiple of 128, so that the groups of
// a warp start on different shared-memory banks.
size_t group_slice(size_t raw, int L) {
    const size_t shift = (size_t)(8 * L) % 128;
    return ((raw + 128 - shift + 127) & ~(size_t)127) - 128 + shift;
}

// One-warp blocks an SM holds: the register cap of the kernel's launch bounds
// and shared memory (1 KB reserved per block).
int packed_resident(size_t smem, int R) {
    const size_t sm_bytes = 228 * 1024;
    const int by_smem = smem + 1024 > sm_bytes ? 0 : (int)(sm_bytes / (smem + 1024));
    return std::min(by_smem, bbs::packed_min_blocks(R));
}

// Reads pattern p's row pointers (the ELL width k is its longest row) and
// picks its class; a pattern whose row pointers do not ascend within
// [0, nnz] is rejected.
bbs_status decide_pattern(const bbs_var_batch* vb, int p, int n, int nnz, int64_t rp_off, int optin,
                          PatPack& pp) {
    std::vector<int32_t> rp(n + 1);
    cudaError_t e = cudaMemcpy(rp.data(), vb->row_ptrs + rp_off, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "pattern row pointers");
    int k = 0;
    for (int r = 0; r < n; ++r) {
        if (rp[r] < 0 || rp[r + 1] < rp[r] || rp[r + 1] > nnz)
            return errf(BBS_ERR_INVALID_ARG, "pattern %d: row pointers must ascend within [0, nnz]", p);
        k = std::max(k, rp[r + 1] - rp[r]);
    }
    pp.state = 2;
    const int n_pad = (n + 1) & ~1;
    for (int L = 4; L <= 16; L *= 2) {
        const int R = (n + L - 1) / L;
        if (R > bbs::kMaxPackedR) continue;
        const size_t raw = align16((size_t)2 * n_pad * 8) + align16((size_t)k * n * 8);
        const size_t smem = group_slice(raw, L) * (size_t)(32 / L);
        if (smem > (size_t)optin || packed_resident(smem, R) < kVarPackedMinWarps) continue;
        pp.state = 1;
        pp.L = L;
        pp.R = R;
        pp.k = k;
        pp.raw = raw;
        break;
    }
    return BBS_OK;
}

// Warps an SM holds of wide blocks of w warps: the kernel may use 255
// registers a thread (8 / w blocks), and shared memory (1 KB reserved per
// block). A wide team is chosen only where this keeps at least the 8 warps a
// persistent block holds: with fewer, the FP64 pipe idles more than the
// saved barriers gain (measured on GB300 with 2D 9-point systems).
int wide_resident_warps(size_t smem, int w) {
    const size_t sm_bytes = 228 * 1024;
    const int by_smem = smem + 1024 > sm_bytes ? 0 : (int)(sm_bytes / (smem + 1024));
    return std::min(by_smem, 8 / w) * w;
}

bbs_status plan_fail(bbs_var_plan* pl, bbs_status s) {
    bbs_var_plan_destroy(pl);
    return s;
}

bbs_status build_plan(bbs_handle* h, const PlanInputs& in, bbs_var_plan** out) {
    const bbs_var_batch* vb = in.vb;
    const bbs_var_tuning& t = in.t;
    const int rmax = t.block_warps == 8 ? 8 : 4;
    const int nb = in.subset ? in.nsubset : vb->num_batch;
    std::vector<int> sys(nb);
    for (int i = 0; i < nb; ++i) sys[i] = in.subset ? in.subset[i] : i;
    const int dev = bbs::handle_device(h);
    int sms = 0, optin = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);

    const int B = t.num_buckets;
    std::vector<int> bucket(nb);
    std::vector<double> cost(nb);
    for (int i = 0; i < nb; ++i) {
        const int p = in.host->sys_pattern[sys[i]];
        const int n = in.host->pat_n[p];
        int b = 0;
        while (b < B && n > t.bucket_max_n[b]) ++b;
        if (b == B) return errf(BBS_ERR_INVALID_ARG, "system %d (n = %d) exceeds the last bucket", sys[i], n);
        bucket[i] = b;
        const double nn = n, nz = in.host->pat_nnz[p];
        cost[i] = (2.0 * nz + 14.0 * nn) * std::sqrt(nn);
    }

    // which systems run packed (their bucket allows it and their pattern's group fits)
    std::vector<PatPack> pat(vb->num_patterns);
    std::vector<int64_t> rp_off;
    std::vector<char> packed(nb, 0);
    for (int i = 0; i < nb; ++i) {
        const int p = in.host->sys_pattern[sys[i]];
        const int n = in.host->pat_n[p];
        if (!t.pack[bucket[i]] || n > kVarPackMaxN) continue;
        if (pat[p].state == 0) {
            if (rp_off.empty()) {
                rp_off.resize(vb->num_patterns);
                cudaError_t e = cudaMemcpy(rp_off.data(), vb->pat_rp_off, sizeof(int64_t) * vb->num_patterns,
                                           cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) return cuda_err(e, "pattern offsets");
            }
            bbs_status s = decide_pattern(vb, p, n, in.host->pat_nnz[p], rp_off[p], optin, pat[p]);
            if (s != BBS_OK) return s;
        }
        packed[i] = pat[p].state == 1;
    }
    // which of the others run as wide teams: a bucket marked wide, BiCGSTAB with
    // Jacobi, more than 8 rows per thread on the fewest warps that keep them
    // within kVarWideMaxR, and a block area that fits
    std::vector<int> wide_w(nb, 0), wide_r(nb, 0);
    const bool wide_ok = in.o->solver == BBS_SOLVER_BICGSTAB && in.o->precond == BBS_PREC_JACOBI;
    std::vector<int> team;
    for (int i = 0; i < nb; ++i) {
        if (packed[i]) continue;
        const int p = in.host->sys_pattern[sys[i]];
        const int n = in.host->pat_n[p];
        // wide bit 1: rows of at most 4 stored values on average; bit 2: denser
        const int density_bit = in.host->pat_nnz[p] <= 4 * n ? 1 : 2;
        if (wide_ok && (t.wide[bucket[i]] & density_bit)) {
            const int w = pow2_at_least((n + 32 * bbs::kVarWideMaxR - 1) / (32 * bbs::kVarWideMaxR));
            const int R = (n + 32 * w - 1) / (32 * w);
            const size_t smem = bbs::varwide_smem(n, in.host->pat_nnz[p]);
            if (w <= 4 && R >= bbs::kVarWideMinR && smem <= (size_t)optin && wide_resident_warps(smem, w) >= 8) {
                wide_w[i] = w;
                wide_r[i] = R;
                continue;
            }
        }
        team.push_back(i);
    }

    // team warps per bucket: at least what the rows need, never more than a larger bucket's
    std::vector<int> nmax(B, 0), W(B);
    for (int i : team) nmax[bucket[i]] = std::max(nmax[bucket[i]], in.host->pat_n[in.host->sys_pattern[sys[i]]]);
    for (int b = 0; b < B; ++b) {
        const int need = pow2_at_least((std::max(nmax[b], 1) + 32 * rmax - 1) / (32 * rmax));
        W[b] = std::max(t.team_warps[b], need);
    }
    for (int b = B - 2; b >= 0; --b) W[b] = std::min(W[b], W[b + 1]);
    for (int b = 0; b < B; ++b)
        if (W[b] > t.block_warps)
            return errf(BBS_ERR_UNSUPPORTED, "bucket %d needs %d warps per system, the block has %d", b, W[b],
                        t.block_warps);

    // team order: team size descending, staging, then estimated cost descending
    std::vector<int> idx = team;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) {
        const int wa = W[bucket[a]], wc = W[bucket[c]];
        if (wa != wc) return wa > wc;
        const int sa = t.stage_values[bucket[a]], sc = t.stage_values[bucket[c]];
        if (sa != sc) return sa > sc;
        return cost[a] > cost[c];
    });

    bbs_var_plan* pl = new bbs_var_plan();
    pl->device = dev;
    pl->num_batch = nb;
    bbs::VarParams& P = pl->P;
    P.num_segments = 0;
    std::vector<int32_t> order;
    order.reserve(nb);
    std::vector<int> seg_nmax, seg_nnzmax;
    for (int k = 0; k < (int)idx.size(); ++k) {
        const int i = idx[k];
        order.push_back(sys[i]);
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
    pl->team_count = (int)idx.size();

    // packed classes, each ordered by estimated cost (similar systems share a warp)
    std::map<std::pair<int, int>, std::vector<int>> cls;
    for (int i = 0; i < nb; ++i)
        if (packed[i]) {
            const PatPack& pp = pat[in.host->sys_pattern[sys[i]]];
            cls[{pp.L, pp.R}].push_back(i);
        }
    std::vector<int> class_begin;
    for (auto& kv : cls) {
        std::vector<int>& m = kv.second;
        std::stable_sort(m.begin(), m.end(), [&](int a, int c) { return cost[a] > cost[c]; });
        class_begin.push_back((int)order.size());
        PackedClass c;
        c.L = kv.first.first;
        c.R = kv.first.second;
        size_t raw = 16;
        for (int i : m) {
            order.push_back(sys[i]);
            raw = std::max(raw, pat[in.host->sys_pattern[sys[i]]].raw);
        }
        c.P.count = (int)m.size();
        c.P.slice = (int)group_slice(raw, c.L);
        c.smem = (size_t)c.P.slice * (size_t)(32 / c.L);
        c.grid = (c.P.count + 32 / c.L - 1) / (32 / c.L);
        c.fn = bbs::varpacked_fn(in.o->solver == BBS_SOLVER_CG ? 1 : 0, c.L, c.R);
        pl->packed_count += c.P.count;
        pl->classes.push_back(c);
    }
    // wide classes, each ordered by estimated cost (longest first)
    std::map<std::pair<int, int>, std::vector<int>> wcls;
    for (int i = 0; i < nb; ++i)
        if (wide_w[i] > 0) wcls[{wide_w[i], wide_r[i]}].push_back(i);
    std::vector<int> wide_begin;
    for (auto& kv : wcls) {
        std::vector<int>& m = kv.second;
        std::stable_sort(m.begin(), m.end(), [&](int a, int c) { return cost[a] > cost[c]; });
        wide_begin.push_back((int)order.size());
        WideClass c;
        c.warps = kv.first.first;
        c.R = kv.first.second;
        for (int i : m) {
            order.push_back(sys[i]);
            const int p = in.host->sys_pattern[sys[i]];
            c.smem = std::max(c.smem, bbs::varwide_smem(in.host->pat_n[p], in.host->pat_nnz[p]));
        }
        c.P.count = (int)m.size();
        c.fn = bbs::varwide_fn(c.R);
        pl->wide_count += c.P.count;
        pl->wides.push_back(c);
    }
    pl->has_team = pl->team_count > 0 || (pl->classes.empty() && pl->wides.empty());

    cudaError_t e;
    if (pl->has_team) {
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
        if (pl->smem > (size_t)optin) {
            delete pl;
            return errf(BBS_ERR_UNSUPPORTED, "the plan needs %zu bytes of shared memory per block (max %d)",
                        pl->smem, optin);
        }
        pl->fn = rmax == 8 ? bbs::varsize_kernel8_fn() : bbs::varsize_kernel4_fn();
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
    }
    for (auto& c : pl->classes)
        if ((e = cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem)) !=
            cudaSuccess)
            return plan_fail(pl, cuda_err(e, "cudaFuncSetAttribute (packed)"));
    for (auto& c : pl->wides)
        if ((e = cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem)) !=
            cudaSuccess)
            return plan_fail(pl, cuda_err(e, "cudaFuncSetAttribute (wide)"));

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
        (e = cudaMalloc(&pl->d_counters, sizeof(int32_t) * bbs::kMaxSeg)) != cudaSuccess)
        return plan_fail(pl, errf(BBS_ERR_NO_MEMORY, "plan buffers: %s", cudaGetErrorString(e)));
    if (nb > 0 && (e = cudaMemcpy(pl->d_order, order.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice)) !=
                      cudaSuccess)
        return plan_fail(pl, cuda_err(e, "order upload"));
    P.order = pl->d_order;
    P.counters = pl->d_counters;
    for (size_t c = 0; c < pl->wides.size(); ++c) {
        bbs::VarWideParams& Q = pl->wides[c].P;
        Q.pat_n = vb->pat_n;
        Q.pat_nnz = vb->pat_nnz;
        Q.rp_off = vb->pat_rp_off;
        Q.ci_off = vb->pat_ci_off;
        Q.row_ptrs = vb->row_ptrs;
        Q.col_idxs = vb->col_idxs;
        Q.sys_pattern = vb->sys_pattern;
        Q.val_off = vb->val_off;
        Q.vec_off = vb->vec_off;
        Q.values = vb->values;
        Q.order = pl->d_order + wide_begin[c];
        Q.cfg = P.cfg;
    }

    if (!pl->classes.empty()) {
        // ELL tables of the packed patterns, built on the device once
        std::vector<int64_t> tab_off(vb->num_patterns, 0);
        std::vector<int32_t> tab_k(vb->num_patterns, 0);
        int64_t total = 0;
        for (int p = 0; p < vb->num_patterns; ++p)
            if (pat[p].state == 1) {
                tab_off[p] = total;
                tab_k[p] = pat[p].k;
                total += (int64_t)pat[p].k * in.host->pat_n[p];
            }
        if ((e = cudaMalloc(&pl->d_tables, sizeof(int32_t) * (size_t)(4 + 2 * total))) != cudaSuccess ||
            (e = cudaMalloc(&pl->d_tab_off, sizeof(int64_t) * vb->num_patterns)) != cudaSuccess ||
            (e = cudaMalloc(&pl->d_tab_k, sizeof(int32_t) * vb->num_patterns)) != cudaSuccess)
            return plan_fail(pl, errf(BBS_ERR_NO_MEMORY, "packed tables: %s", cudaGetErrorString(e)));
        if ((e = cudaMemcpy(pl->d_tab_off, tab_off.data(), sizeof(int64_t) * vb->num_patterns,
                            cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(pl->d_tab_k, tab_k.data(), sizeof(int32_t) * vb->num_patterns,
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return plan_fail(pl, cuda_err(e, "packed table upload"));
        int32_t* flag = pl->d_tables;
        int32_t* xcols = pl->d_tables + 4;
        int32_t* xsrc = xcols + total;
        cudaStream_t st;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
            return plan_fail(pl, cuda_err(e, "table stream"));
        std::vector<int64_t> ci_off(vb->num_patterns);
        e = cudaMemcpy(ci_off.data(), vb->pat_ci_off, sizeof(int64_t) * vb->num_patterns, cudaMemcpyDeviceToHost);
        for (int p = 0; p < vb->num_patterns && e == cudaSuccess; ++p)
            if (pat[p].state == 1 && pat[p].k > 0)
                e = bbs::launch_csr_ell_tables(in.host->pat_n[p], pat[p].k, vb->row_ptrs + rp_off[p],
                                               vb->col_idxs + ci_off[p], xcols + tab_off[p], xsrc + tab_off[p],
                                               flag, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
        if (e != cudaSuccess) return plan_fail(pl, cuda_err(e, "packed tables"));
        for (size_t c = 0; c < pl->classes.size(); ++c) {
            bbs::VarPackedParams& Q = pl->classes[c].P;
            Q.pat_n = vb->pat_n;
            Q.rp_off = vb->pat_rp_off;
            Q.ci_off = vb->pat_ci_off;
            Q.row_ptrs = vb->row_ptrs;
            Q.col_idxs = vb->col_idxs;
            Q.sys_pattern = vb->sys_pattern;
            Q.val_off = vb->val_off;
            Q.vec_off = vb->vec_off;
            Q.values = vb->values;
            Q.tab_off = pl->d_tab_off;
            Q.tab_k = pl->d_tab_k;
            Q.xcols = xcols;
            Q.xsrc = xsrc;
            Q.order = pl->d_order + class_begin[c];
            Q.cfg = P.cfg;
        }
    }

    // graph: [reset the work counters -> the persistent launch] beside one
    // launch per packed class and per wide class (no order among them)
    if ((e = cudaGraphCreate(&pl->graph, 0)) != cudaSuccess) return plan_fail(pl, cuda_err(e, "graph create"));
    if (pl->has_team) {
        cudaMemsetParams mp{};
        mp.dst = pl->d_counters;
        mp.elementSize = sizeof(int32_t);
        mp.width = bbs::kMaxSeg;
        mp.height = 1;
        mp.value = 0;
        mp.pitch = 0;
        cudaGraphNode_t mset = nullptr;
        if ((e = cudaGraphAddMemsetNode(&mset, pl->graph, nullptr, 0, &mp)) != cudaSuccess)
            return plan_fail(pl, cuda_err(e, "graph memset node"));
        void* args[] = {&P};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(pl->fn);
        kp.gridDim = dim3(pl->grid);
        kp.blockDim = dim3(pl->threads);
        kp.sharedMemBytes = (unsigned)pl->smem;
        kp.kernelParams = args;
        if ((e = cudaGraphAddKernelNode(&pl->knode, pl->graph, &mset, 1, &kp)) != cudaSuccess)
            return plan_fail(pl, cuda_err(e, "graph kernel node"));
    }
    for (auto& c : pl->classes) {
        void* args[] = {&c.P};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(c.fn);
        kp.gridDim = dim3(c.grid);
        kp.blockDim = dim3(32);
        kp.sharedMemBytes = (unsigned)c.smem;
        kp.kernelParams = args;
        if ((e = cudaGraphAddKernelNode(&c.node, pl->graph, nullptr, 0, &kp)) != cudaSuccess)
            return plan_fail(pl, cuda_err(e, "graph packed node"));
    }
    for (auto& c : pl->wides) {
        void* args[] = {&c.P};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(c.fn);
        kp.gridDim = dim3(c.P.count);
        kp.blockDim = dim3(32 * c.warps);
        kp.sharedMemBytes = (unsigned)c.smem;
        kp.kernelParams = args;
        if ((e = cudaGraphAddKernelNode(&c.node, pl->graph, nullptr, 0, &kp)) != cudaSuccess)
            return plan_fail(pl, cuda_err(e, "graph wide node"));
    }
    if ((e = cudaGraphInstantiate(&pl->exec, pl->graph, 0)) != cudaSuccess)
        return plan_fail(pl, cuda_err(e, "graph instantiate"));
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
        t->pack[b] = 1;
        // measured on GB300: wide teams pay above 512 rows for 3-point rows
        // (18 % faster), not for 5- and 9-point rows, nor at 512 rows or less
        t->wide[b] = e > 512 ? 1 : 0;
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
    cudaError_t e;
    if (pl->has_team) {
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
        if ((e = cudaGraphExecKernelNodeSetParams(pl->exec, pl->knode, &kp)) != cudaSuccess)
            return cuda_err(e, "graph parameter update");
    }
    for (auto& c : pl->classes) {
        c.P.b = b;
        c.P.x = x;
        c.P.iters = log->iters;
        c.P.rel_res = log->rel_res;
        c.P.status = log->status;
        void* args[] = {&c.P};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(c.fn);
        kp.gridDim = dim3(c.grid);
        kp.blockDim = dim3(32);
        kp.sharedMemBytes = (unsigned)c.smem;
        kp.kernelParams = args;
        if ((e = cudaGraphExecKernelNodeSetParams(pl->exec, c.node, &kp)) != cudaSuccess)
            return cuda_err(e, "graph parameter update (packed)");
    }
    for (auto& c : pl->wides) {
        c.P.b = b;
        c.P.x = x;
        c.P.iters = log->iters;
        c.P.rel_res = log->rel_res;
        c.P.status = log->status;
        void* args[] = {&c.P};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(c.fn);
        kp.gridDim = dim3(c.P.count);
        kp.blockDim = dim3(32 * c.warps);
        kp.sharedMemBytes = (unsigned)c.smem;
        kp.kernelParams = args;
        if ((e = cudaGraphExecKernelNodeSetParams(pl->exec, c.node, &kp)) != cudaSuccess)
            return cuda_err(e, "graph parameter update (wide)");
    }
    if ((e = cudaGraphLaunch(pl->exec, reinterpret_cast<cudaStream_t>(stream))) != cudaSuccess)
        return cuda_err(e, "graph launch");
    return BBS_OK;
}

bbs_status bbs_var_plan_describe(const bbs_var_plan* pl, bbs_var_plan_desc* d) {
    if (pl == nullptr || d == nullptr) return errf(BBS_ERR_INVALID_ARG, "null plan or description");
    d->team_systems = pl->team_count;
    d->packed_systems = pl->packed_count;
    d->packed_launches = (int32_t)pl->classes.size();
    d->wide_systems = pl->wide_count;
    d->wide_launches = (int32_t)pl->wides.size();
    d->persistent_grid = pl->has_team ? pl->grid : 0;
    return BBS_OK;
}

bbs_status bbs_var_plan_destroy(bbs_var_plan* pl) {
    if (pl == nullptr) return BBS_OK;
    cudaSetDevice(pl->device);
    cudaDeviceSynchronize();
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->d_order) cudaFree(pl->d_order);
    if (pl->d_counters) cudaFree(pl->d_counters);
    if (pl->d_tables) cudaFree(pl->d_tables);
    if (pl->d_tab_off) cudaFree(pl->d_tab_off);
    if (pl->d_tab_k) cudaFree(pl->d_tab_k);
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

    // per-system time of a plan of the systems `sys` (INFINITY if the
    // choice cannot be planned)
    auto time_plan = [&](const bbs_var_tuning& t, const std::vector<int>& sys) -> double {
        PlanInputs in{vb, host, o, t, sys.data(), (int)sys.size()};
        bbs_var_plan* pl = nullptr;
        if (build_plan(h, in, &pl) != BBS_OK) return INFINITY;
        float ms_sum = 0.f;
        bool ok = true;
        // one untimed run, then at least three timed ones and until 10 ms
        // are timed (a small bucket's trial takes a fraction of a
        // millisecond, where one run's noise exceeds the margins below)
        int timed = 0;
        for (int rep = 0; ok && (rep < 4 || (ms_sum < 10.f && rep < 64)); ++rep) {
            cudaMemcpyAsync(dx, x0, sizeof(double) * vec_len, cudaMemcpyDeviceToDevice, st);
            cudaEventRecord(e0, st);
            ok = bbs_var_solve(pl, b, dx, &lg, st) == BBS_OK;
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) {
                ms_sum += ms;
                ++timed;
            }
        }
        bbs_var_plan_destroy(pl);
        return ok ? ms_sum / timed / sys.size() : INFINITY;
    };
    // one launch choice on bucket k's sample alone
    auto trial = [&](int k, int bw, int w, int stg, int pack, int wide) -> double {
        bbs_var_tuning t;
        std::memset(&t, 0, sizeof t);
        t.num_buckets = 1;
        t.bucket_max_n[0] = 2048;
        t.team_warps[0] = w;
        t.stage_values[0] = stg;
        t.pack[0] = pack;
        t.wide[0] = wide;
        t.block_warps = bw;
        return time_plan(t, samp[k]);
    };
    std::vector<int> all_samples;
    std::vector<char> has_small(B, 0);
    for (int k = 0; k < B; ++k) {
        all_samples.insert(all_samples.end(), samp[k].begin(), samp[k].end());
        for (int i : samp[k])
            if (host->pat_n[host->sys_pattern[i]] <= kVarPackMaxN) has_small[k] = 1;
    }

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
            int nk = 0, nmin = 1 << 30;
            for (int i : samp[k]) {
                nk = std::max(nk, host->pat_n[host->sys_pattern[i]]);
                nmin = std::min(nmin, host->pat_n[host->sys_pattern[i]]);
            }
            const int wmin = pow2_at_least((nk + 32 * rmax - 1) / (32 * rmax));
            double best = INFINITY;
            int bestw = wmin, bests = 0, bestp = 0;
            for (int w = wmin; w <= bw; w *= 2)
                for (int stg = 0; stg <= 1; ++stg) {
                    const double per = trial(k, bw, w, stg, 0, 0);
                    if (per < best) {
                        best = per;
                        bestw = w;
                        bests = stg;
                    }
                }
            // Packing the bucket's small systems (the rest as the best team
            // choice), then wide teams for its systems that need more than 8
            // rows per thread on their fewest warps. Each is kept or dropped
            // against the default tuning's choice, which the trial must beat
            // by 3 % to be overturned: near-equal trials then give the same
            // plan from run to run, and a packed class timed alone (it runs
            // beside the other launches in a full plan) is not counted against
            // packing for a difference of a percent or two.
            const auto prefer = [](double alt, double cur, bool alt_is_default) {
                return alt_is_default ? alt <= cur * 1.03 : alt < cur * 0.97;
            };
            if (nmin <= kVarPackMaxN) {
                const double per = trial(k, bw, bestw, bests, 1, 0);
                if (prefer(per, best, base.pack[k] != 0)) {
                    best = per;
                    bestp = 1;
                }
            }
            int bestwide = 0;
            if (o->solver == BBS_SOLVER_BICGSTAB && o->precond == BBS_PREC_JACOBI && nk > 32 * 8) {
                for (int bit : {1, 2}) {  // sparse rows, then denser rows
                    const double per = trial(k, bw, bestw, bests, bestp, bestwide | bit);
                    if (prefer(per, best, (base.wide[k] & bit) != 0)) {
                        best = per;
                        bestwide |= bit;
                    }
                }
            }
            if (!std::isfinite(best)) {
                feasible = false;
                break;
            }
            cand.team_warps[k] = bestw;
            cand.stage_values[k] = bests;
            cand.pack[k] = bestp;
            cand.wide[k] = bestwide;
            total += best * members[k].size();
        }
        // Packed classes and wide teams run beside the persistent launch in a
        // full plan, which a bucket timed alone does not show. The sample of
        // the whole batch (the real plan's shape, so a 1 % margin) decides
        // two things: where the buckets' trials left small systems unpacked
        // against the default, whether to pack them after all; and where wide
        // teams are on, whether to keep them.
        if (feasible) {
            double t_cand = -1.0;
            bbs_var_tuning packed = cand;
            bool differs = false;
            for (int k = 0; k < B; ++k)
                if (has_small[k] && base.pack[k] && !cand.pack[k]) {
                    packed.pack[k] = 1;
                    differs = true;
                }
            if (differs) {
                t_cand = time_plan(cand, all_samples);
                const double t_packed = time_plan(packed, all_samples);
                if (std::isfinite(t_packed) && t_packed <= t_cand * 1.01) {
                    cand = packed;
                    t_cand = t_packed;
                }
            }
            bbs_var_tuning narrow = cand;
            differs = false;
            for (int k = 0; k < B; ++k)
                if (cand.wide[k]) {
                    narrow.wide[k] = 0;
                    differs = true;
                }
            if (differs) {
                if (t_cand < 0.0) t_cand = time_plan(cand, all_samples);
                const double t_narrow = time_plan(narrow, all_samples);
                if (std::isfinite(t_narrow) && t_narrow < t_cand * 0.99) cand = narrow;
            }
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
