// Batched solve: many problems of uneven size, each with its own Theta_K, blur and lambda,
// advanced together. Every iteration is two launches that cover the tiles of every running
// problem (heaviest tiles first across all problems, persistent CTAs pulling from one
// queue); a problem that meets its own stopping rule drops out of the queue. Chunks of
// check_every iterations are captured in a CUDA graph and replayed until no problem runs;
// between chunks the host compacts the two work lists to the problems still running (the
// kernels read the item counts from device memory, so the captured graph stays valid).
// The tiles come from each operator's batch plans, whose tile sides are the autotuner's and
// whose items are grouped (one item per level and tile covers every subband of the level).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <set>

#include "solve_impl.h"
#include "theta_impl.h"
#include "tile.cuh"

namespace wdb {

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct DevBuf {
    std::vector<void*> ptrs;
    ~DevBuf() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    wdb_status alloc(T** p, size_t n) {
        void* q = nullptr;
        WDB_CK(cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)));
        ptrs.push_back(q);
        *p = static_cast<T*>(q);
        return WDB_OK;
    }
};

std::vector<BatchItem> merge_items(const std::vector<wdb_theta*>& th, int op) {
    struct C {
        BatchItem it;
        double cost;
    };
    std::vector<C> all;
    for (int p = 0; p < (int)th.size(); ++p) {
        const TilePlanHost& h = th[p]->bplan[op];
        for (int i = 0; i < (int)h.items.size(); ++i) all.push_back({BatchItem{p, i}, h.item_cost[i]});
    }
    std::stable_sort(all.begin(), all.end(), [](const C& a, const C& b) { return a.cost > b.cost; });
    std::vector<BatchItem> out(all.size());
    for (size_t i = 0; i < all.size(); ++i) out[i] = all[i].it;
    return out;
}

}  // namespace

wdb_status solve_batch(int B, wdb_theta* const* ths, const float* const* u, float* const* x,
                       const wdb_solve_params* params, cudaStream_t caller, wdb_solve_result* res) {
    const double t0 = now_ms();
    if (B < 1) return set_error(WDB_EINVAL, "batch size must be >= 1");
    if (!ths || !u || !x || !params || !res) return set_error(WDB_EINVAL, "NULL argument");
    std::vector<wdb_theta*> th(ths, ths + B);
    std::set<wdb_theta*> uniq(th.begin(), th.end());
    if ((int)uniq.size() != B || uniq.count(nullptr)) return set_error(WDB_EINVAL, "every problem needs its own handle");
    int m = 0;
    for (int b = 0; b < B; ++b) {
        if (!u[b] || !x[b]) return set_error(WDB_EINVAL, "NULL buffer for problem %d", b);
        const wdb_solve_params& p = params[b];
        if (p.max_iters < 1 || !(p.tol >= 0.0) || p.precond < 0 || p.precond > 2 || !std::isfinite(p.target_objective))
            return set_error(WDB_EINVAL, "bad parameters for problem %d", b);
        const int mb = p.check_every > 0 ? p.check_every : 10;
        if (b == 0) m = mb;
        else if (mb != m) return set_error(WDB_EINVAL, "all problems of a batch share check_every");
    }
    WDB_TRY(work_enter(&th[0]->work, &th[0]->ev_in, &th[0]->ev_out, caller));
    cudaStream_t st = th[0]->work;
    // Every return from here on makes the caller's stream wait for the work queued so far
    // (so that a caller reusing its buffers after an error does not race with it) and
    // releases the pinned flag; the successful path rejoins explicitly and checks for errors.
    struct Rejoin {
        cudaStream_t work, caller;
        cudaEvent_t ev;
        int* pinned = nullptr;
        bool done = false;
        ~Rejoin() {
            if (!done) {
                cudaEventRecord(ev, work);
                cudaStreamWaitEvent(caller, ev, 0);
            }
            if (pinned) {
                cudaStreamSynchronize(work);
                cudaFreeHost(pinned);
            }
        }
    } rejoin{st, caller, th[0]->ev_out};
    // per-problem set-up: preconditioner, workspace, x0 = Psi* u, weights, start, state
    std::vector<BatchProblem> hp(B);
    int buf_elems = 16;
    for (int b = 0; b < B; ++b) {
        wdb_theta* t = th[b];
        const wdb_solve_params& p = params[b];
        WDB_TRY(theta_precond(t, p.precond, p.jacobi_eps, st));
        WDB_TRY(theta_workspace_public(t, st));
        const long long N = t->lay.N;
        WDB_TRY(dwt2<float>(u[b], t->d_x0, t->lay, t->filt, t->d_scr, st));
        std::vector<float> w(t->lay.S);
        for (int s = 0; s < t->lay.S; ++s) w[s] = (float)(p.w_subband_host ? p.w_subband_host[s] : p.lambda);
        WDB_CK(cudaMemcpyAsync(t->d_w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, st));
        if (p.x_init_dev) {
            WDB_CK(cudaMemcpyAsync(t->d_xs, p.x_init_dev, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
            WDB_CK(cudaMemcpyAsync(t->d_y, p.x_init_dev, sizeof(float) * N, cudaMemcpyDeviceToDevice, st));
        } else {
            WDB_CK(cudaMemsetAsync(t->d_xs, 0, sizeof(float) * N, st));
            WDB_CK(cudaMemsetAsync(t->d_y, 0, sizeof(float) * N, st));
        }
        SolveState s0;
        std::memset(&s0, 0, sizeof s0);
        s0.k = 1;
        s0.max_iters = p.max_iters;
        s0.check_every = m;
        s0.tol = p.tol;
        s0.primal = s0.dual = s0.gap = s0.rel_gap = NAN;
        s0.target = p.target_objective > 0.0 ? p.target_objective : 0.0;
        s0.ista = p.ista ? 1 : 0;
        WDB_CK(cudaMemcpyAsync(t->d_state, &s0, sizeof s0, cudaMemcpyHostToDevice, st));
        BatchProblem& q = hp[b];
        WDB_TRY(theta_batch_plans(t, st));
        q.fwd = t->bargs[0].plan;
        q.adj = t->bargs[1].plan;
        q.sb = t->d_sb;
        q.y = t->d_y;
        q.x = t->d_xs;
        q.r = t->d_r;
        q.x0 = t->d_x0;
        q.step_tab = t->pc[p.precond].d_step;
        q.w_sb = t->d_w;
        q.st = t->d_state;
        q.sums = nullptr;
        buf_elems = std::max({buf_elems, q.fwd.buf_elems, q.adj.buf_elems});
    }
    DevBuf mem;
    double* d_sums = nullptr;
    BatchProblem* d_probs = nullptr;
    BatchItem *d_fwd = nullptr, *d_adj = nullptr;
    TileQueue* d_q = nullptr;
    int* d_running = nullptr;
    int* d_counts = nullptr;       // item counts of the two phases (compacted between chunks)
    int* d_flags = nullptr;        // per problem: still running
    WDB_TRY(mem.alloc(&d_sums, 4 * (size_t)B));
    for (int b = 0; b < B; ++b) hp[b].sums = d_sums + 4 * b;
    const std::vector<BatchItem> fi = merge_items(th, 0), ai = merge_items(th, 1);
    WDB_TRY(mem.alloc(&d_probs, B));
    WDB_TRY(mem.alloc(&d_fwd, fi.size()));
    WDB_TRY(mem.alloc(&d_adj, ai.size()));
    WDB_TRY(mem.alloc(&d_q, 1));
    WDB_TRY(mem.alloc(&d_running, 1));
    WDB_TRY(mem.alloc(&d_counts, 2));
    WDB_TRY(mem.alloc(&d_flags, B));
    WDB_CK(cudaMemsetAsync(d_sums, 0, sizeof(double) * 4 * B, st));
    WDB_CK(cudaMemsetAsync(d_q, 0, sizeof(TileQueue), st));
    WDB_CK(cudaMemcpyAsync(d_probs, hp.data(), sizeof(BatchProblem) * B, cudaMemcpyHostToDevice, st));
    WDB_CK(cudaMemcpyAsync(d_fwd, fi.data(), sizeof(BatchItem) * fi.size(), cudaMemcpyHostToDevice, st));
    WDB_CK(cudaMemcpyAsync(d_adj, ai.data(), sizeof(BatchItem) * ai.size(), cudaMemcpyHostToDevice, st));
    int h_counts[2] = {(int)fi.size(), (int)ai.size()};
    WDB_CK(cudaMemcpyAsync(d_counts, h_counts, sizeof h_counts, cudaMemcpyHostToDevice, st));
    int* h_running = nullptr;
    WDB_CK(cudaMallocHost(&h_running, sizeof(int)));
    rejoin.pinned = h_running;
    *h_running = B;
    BatchArgs F{}, A{};
    F.probs = A.probs = d_probs;
    F.B = A.B = B;
    F.items = d_fwd;
    F.n_items = (int)fi.size();
    A.items = d_adj;
    A.n_items = (int)ai.size();
    F.queue = A.queue = d_q;
    F.running = A.running = d_running;
    F.run_flags = A.run_flags = d_flags;
    F.n_items_dev = d_counts;
    A.n_items_dev = d_counts + 1;
    F.buf_elems = A.buf_elems = buf_elems;
    F.smem_bytes = A.smem_bytes = 2 * buf_elems * (int)sizeof(float);
    bool grouped = false;
    for (int b = 0; b < B; ++b) grouped = grouped || hp[b].fwd.n_grp > 0 || hp[b].adj.n_grp > 0;
    F.grouped = A.grouped = grouped ? 1 : 0;
    F.grid = A.grid = std::max(1, tile_batch_grid(F.smem_bytes, grouped));
    // chunks of m iterations in a CUDA graph, replayed until no problem is running
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    wdb_status s = WDB_OK;
    cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) s = cuda_error(ce, "begin capture", __FILE__, __LINE__);
    for (int i = 0; i < m && s == WDB_OK; ++i) {
        s = batch_k1(F, st);
        if (s == WDB_OK) s = batch_k2(A, st);
    }
    if (s == WDB_OK) {
        ce = cudaMemcpyAsync(h_running, d_running, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (ce != cudaSuccess) s = cuda_error(ce, "capture copy", __FILE__, __LINE__);
    }
    ce = cudaStreamEndCapture(st, &g);
    if (s == WDB_OK && ce != cudaSuccess) s = cuda_error(ce, "end capture", __FILE__, __LINE__);
    if (s == WDB_OK) {
        ce = cudaGraphInstantiate(&ge, g, 0);
        if (ce != cudaSuccess) s = cuda_error(ce, "instantiate", __FILE__, __LINE__);
    }
    if (g) cudaGraphDestroy(g);
    count_launch(-2LL * m);
    int max_it = 0;
    for (int b = 0; b < B; ++b) max_it = std::max(max_it, params[b].max_iters);
    // between chunks the work lists are compacted to the problems still running, so that the
    // launches of a long tail do not walk the tiles of finished problems
    int prev_running = B;
    std::vector<int> flags(B);
    std::vector<BatchItem> cf, ca;
    for (int chunk = 0; s == WDB_OK; ++chunk) {
        ce = cudaGraphLaunch(ge, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) {
            s = cuda_error(ce, "batch chunk", __FILE__, __LINE__);
            break;
        }
        count_launch(2LL * m);
        if (*h_running == 0 || (long long)(chunk + 1) * m >= max_it) break;
        if (*h_running < prev_running) {
            prev_running = *h_running;
            ce = cudaMemcpy(flags.data(), d_flags, sizeof(int) * B, cudaMemcpyDeviceToHost);
            if (ce != cudaSuccess) {
                s = cuda_error(ce, "batch flags", __FILE__, __LINE__);
                break;
            }
            cf.clear();
            ca.clear();
            for (const BatchItem& it : fi)
                if (flags[it.p]) cf.push_back(it);
            for (const BatchItem& it : ai)
                if (flags[it.p]) ca.push_back(it);
            const int hc[2] = {(int)cf.size(), (int)ca.size()};
            ce = cudaMemcpyAsync(d_fwd, cf.data(), sizeof(BatchItem) * std::max<size_t>(cf.size(), 1),
                                 cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(d_adj, ca.data(), sizeof(BatchItem) * std::max<size_t>(ca.size(), 1),
                                     cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_counts, hc, sizeof hc, cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            if (ce != cudaSuccess) {
                s = cuda_error(ce, "batch compaction", __FILE__, __LINE__);
                break;
            }
        }
    }
    if (ge) cudaGraphExecDestroy(ge);
    // exact objective of every returned x (the full work list again)
    if (s == WDB_OK) {
        ce = cudaMemcpyAsync(d_fwd, fi.data(), sizeof(BatchItem) * fi.size(), cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_counts, h_counts, sizeof h_counts, cudaMemcpyHostToDevice, st);
        if (ce != cudaSuccess) s = cuda_error(ce, "batch list", __FILE__, __LINE__);
    }
    if (s == WDB_OK) s = batch_objective(F, st);
    std::vector<double> sums(4 * B);
    std::vector<SolveState> states(B);
    if (s == WDB_OK) {
        ce = cudaMemcpyAsync(sums.data(), d_sums, sizeof(double) * 4 * B, cudaMemcpyDeviceToHost, st);
        for (int b = 0; b < B && ce == cudaSuccess; ++b)
            ce = cudaMemcpyAsync(&states[b], th[b]->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, st);
        for (int b = 0; b < B && ce == cudaSuccess; ++b)
            ce = cudaMemcpyAsync(x[b], th[b]->d_xs, sizeof(float) * th[b]->lay.N, cudaMemcpyDeviceToDevice, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) s = cuda_error(ce, "batch results", __FILE__, __LINE__);
    }
    if (s == WDB_OK) {
        s = work_exit(st, th[0]->ev_out, caller);
        rejoin.done = s == WDB_OK;
    }
    const double ms = now_ms() - t0;
    for (int b = 0; b < B; ++b) {
        wdb_solve_result& r = res[b];
        std::memset(&r, 0, sizeof r);
        r.status = s;
        if (s != WDB_OK) continue;
        const SolveState& q = states[b];
        r.iters = q.iters_done;
        r.objective = 0.5 * sums[4 * b] + sums[4 * b + 1];
        r.primal = q.primal;
        r.gap = q.gap;
        r.rel_gap = q.rel_gap;
        r.support = -1;
        r.tau = th[b]->pc[params[b].precond].tau;
        r.L_hat = th[b]->pc[params[b].precond].L_hat;
        r.solve_ms = ms;
        r.first_primal_below = q.hit_k;
        r.kkt_off = r.kkt_on = r.gap64 = r.rel_gap64 = NAN;
        if (q.nan_flag || !std::isfinite(r.objective)) r.status = set_error(WDB_ENAN, "problem %d: NaN/Inf", b);
        else if (q.diverged) r.status = set_error(WDB_EDIVERGED, "problem %d: objective diverged", b);
    }
    return s;
}

}  // namespace wdb
