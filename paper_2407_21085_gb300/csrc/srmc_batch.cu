// srmc_batch.cu -- the batched form: many independent SRMC instances solved
// together, by one of two strategies captured into one CUDA graph:
//   ROUNDS    instances grouped by kernel variant (d, basis, model variant,
//             control); their backward loops aligned at the end (round s
//             solves step N_r - 1 - s of every instance with N_r > s); each
//             round of each group is one launch of step_kernel_batch over the
//             concatenated strata of its active instances, on a persistent
//             grid.  Parameters come from device memory.
//   BRANCHES  every instance keeps its own single-instance step launches
//             (parameters in the constant bank) on its own branch of the
//             graph, so the launch chains of different instances run
//             concurrently and small instances fill the GPU together.
//   FLOW      one persistent launch per variant group over all of its rounds
//             (step_kernel_flow): blocks take (instance, step, stratum) items
//             in round order from a counter and wait, item by item, only for
//             the previous step of their own instance; the groups' launches
//             run on parallel branches of the graph.
// The tuner picks, per variant group, the threads per stratum block (and the
// blocks per SM for ROUNDS) by timing, then times both strategies on the
// whole batch and keeps the faster.
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/srmc.h"
#include "srmc_internal.h"

namespace {

srmc_status bfail(srmc_status st, const std::string &m)
{
    srmc::set_last_error(m);
    return st;
}

#define BATCH_CUDA(call, what)                                                                 \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return bfail(e_ == cudaErrorMemoryAllocation ? SRMC_ERR_OOM : SRMC_ERR_CUDA,       \
                         std::string(what) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

using LaunchFn = cudaError_t (*)(const srmc::BatchRound &, bool, bool, int, bool, int, int, cudaStream_t);
using OccFn = int (*)(bool, bool, int, bool, int);
using FlowFn = cudaError_t (*)(const srmc::FlowPlan &, bool, int, bool, int, int, cudaStream_t);
using FlowOccFn = int (*)(bool, int, bool, int);

FlowFn flow_for(int d)
{
    switch (d) {
    case 1: return srmc::launch_flow_d1; case 2: return srmc::launch_flow_d2;
    case 3: return srmc::launch_flow_d3; case 4: return srmc::launch_flow_d4;
    case 5: return srmc::launch_flow_d5; case 6: return srmc::launch_flow_d6;
    case 7: return srmc::launch_flow_d7; case 8: return srmc::launch_flow_d8;
    }
    return nullptr;
}

FlowOccFn flow_occ_for(int d)
{
    switch (d) {
    case 1: return srmc::occupancy_flow_d1; case 2: return srmc::occupancy_flow_d2;
    case 3: return srmc::occupancy_flow_d3; case 4: return srmc::occupancy_flow_d4;
    case 5: return srmc::occupancy_flow_d5; case 6: return srmc::occupancy_flow_d6;
    case 7: return srmc::occupancy_flow_d7; case 8: return srmc::occupancy_flow_d8;
    }
    return nullptr;
}

LaunchFn launch_for(int d)
{
    switch (d) {
    case 1: return srmc::launch_batch_d1; case 2: return srmc::launch_batch_d2;
    case 3: return srmc::launch_batch_d3; case 4: return srmc::launch_batch_d4;
    case 5: return srmc::launch_batch_d5; case 6: return srmc::launch_batch_d6;
    case 7: return srmc::launch_batch_d7; case 8: return srmc::launch_batch_d8;
    }
    return nullptr;
}

OccFn occ_for(int d)
{
    switch (d) {
    case 1: return srmc::occupancy_batch_d1; case 2: return srmc::occupancy_batch_d2;
    case 3: return srmc::occupancy_batch_d3; case 4: return srmc::occupancy_batch_d4;
    case 5: return srmc::occupancy_batch_d5; case 6: return srmc::occupancy_batch_d6;
    case 7: return srmc::occupancy_batch_d7; case 8: return srmc::occupancy_batch_d8;
    }
    return nullptr;
}

struct Round {                  // one launch: a group's active instances in round s
    int s;
    int n_active;
    long long total;
    long long off;              // offset of its inst/step arrays in the int buffer
    long long koff;             // offset of its kofs array in the long long buffer
};

struct Group {
    int d, mv;
    bool lp1, cv;
    std::vector<int> members;   // instance indices
    std::vector<Round> rounds;
    int threads = 256;
    int blocks_per_sm = 0;      // 0: occupancy limit
    // FLOW: the group's segments (round order) on the device
    int n_seg = 0;
    long long flow_total = 0;
    int *f_inst = nullptr, *f_step = nullptr, *f_dep = nullptr;
    long long *f_kofs = nullptr;
    unsigned long long *f_done = nullptr;   // [n_seg + 1]: done counters, then the work counter
};

}  // namespace

enum { MODE_ROUNDS = 0, MODE_BRANCHES = 1, MODE_FLOW = 2 };
constexpr int kBranchStreams = 64;

struct srmc_batch {
    std::vector<srmc_solver *> solvers;
    int mode = MODE_ROUNDS;
    std::vector<cudaStream_t> branch;   // capture streams of the BRANCHES strategy
    std::vector<cudaEvent_t> ev;        // fork/join events
    std::vector<Group> groups;
    Params *d_params = nullptr;
    int *d_ints = nullptr;
    long long *d_kofs = nullptr;
    unsigned *d_error = nullptr;        // FLOW: set when a wait gave up
    int sms = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    float strategy_ms[3] = {-1.0f, -1.0f, -1.0f};   // the tuner's timings of the strategies
};

namespace {

void batch_free(srmc_batch *b)
{
    for (auto &g : b->groups) {
        cudaFree(g.f_inst); cudaFree(g.f_step); cudaFree(g.f_dep); cudaFree(g.f_kofs); cudaFree(g.f_done);
    }
    cudaFree(b->d_error);
    for (auto st : b->branch) cudaStreamDestroy(st);
    for (auto e : b->ev) cudaEventDestroy(e);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->d_params);
    cudaFree(b->d_ints);
    cudaFree(b->d_kofs);
}

srmc::BatchRound round_args(const srmc_batch *b, const Round &r)
{
    srmc::BatchRound B;
    B.params = b->d_params;
    B.inst = b->d_ints + r.off;
    B.step = b->d_ints + r.off + r.n_active;
    B.kofs = b->d_kofs + r.koff;
    B.n_active = r.n_active;
    B.total = r.total;
    return B;
}

cudaError_t launch_round(const srmc_batch *b, const Group &g, const Round &r, int threads, int bps,
                         cudaStream_t st)
{
    int occ = occ_for(g.d)(false, g.lp1, g.mv, g.cv, threads);
    if (occ <= 0) return cudaErrorInvalidConfiguration;
    if (bps <= 0 || bps > occ) bps = occ;
    long long grid = (long long)b->sms * bps;
    if (grid > r.total) grid = r.total;
    return launch_for(g.d)(round_args(b, r), false, g.lp1, g.mv, g.cv, (int)grid, threads, st);
}

// BRANCHES: fork onto kBranchStreams streams, instances dealt out in
// decreasing order of work (longest first), each stream's instances one
// after the other, then join.
cudaError_t ensure_streams(srmc_batch *b)
{
    cudaError_t e = cudaSuccess;
    if (b->branch.empty()) {
        for (int a = 0; a < kBranchStreams && e == cudaSuccess; ++a) {
            cudaStream_t x;
            e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
            if (e == cudaSuccess) b->branch.push_back(x);
        }
        for (int a = 0; a < kBranchStreams + 1 && e == cudaSuccess; ++a) {
            cudaEvent_t x;
            e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
            if (e == cudaSuccess) b->ev.push_back(x);
        }
    }
    return e;
}

cudaError_t enqueue_branches(srmc_batch *b, cudaStream_t st)
{
    cudaError_t e = ensure_streams(b);
    if (e != cudaSuccess) return e;
    std::vector<int> order(b->solvers.size());
    for (size_t r = 0; r < order.size(); ++r) order[r] = (int)r;
    auto work = [&](int r) {
        const Params &P = b->solvers[r]->P;
        return (double)b->solvers[r]->M_sum * (double)P.N * (double)(P.N + 1);
    };
    std::sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
    const int ns = (int)std::min<size_t>(b->branch.size(), order.size());
    if ((e = cudaEventRecord(b->ev[kBranchStreams], st)) != cudaSuccess) return e;
    for (int a = 0; a < ns; ++a)
        if ((e = cudaStreamWaitEvent(b->branch[a], b->ev[kBranchStreams], 0)) != cudaSuccess) return e;
    for (size_t q = 0; q < order.size(); ++q) {
        const srmc_solver *s = b->solvers[order[q]];
        cudaStream_t x = b->branch[q % ns];
        for (int i = s->P.N - 1; i >= 0; --i)
            if ((e = srmc_launch_solver_step(s, i, x)) != cudaSuccess) return e;
    }
    for (int a = 0; a < ns; ++a) {
        if ((e = cudaEventRecord(b->ev[a], b->branch[a])) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, b->ev[a], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// FLOW: the group segments in round order (built on first use), then per
// group a cleared counter block and one persistent launch, the groups on
// parallel branches of the graph.
cudaError_t ensure_streams(srmc_batch *b);

cudaError_t build_flow(srmc_batch *b)
{
    cudaError_t e = cudaSuccess;
    if (!b->d_error) {
        if ((e = cudaMalloc(&b->d_error, sizeof(unsigned))) != cudaSuccess) return e;
        if ((e = cudaMemset(b->d_error, 0, sizeof(unsigned))) != cudaSuccess) return e;
    }
    for (auto &g : b->groups) {
        if (g.f_inst) continue;
        std::vector<int> inst, step, dep;
        std::vector<long long> kofs(1, 0);
        std::vector<int> last(b->solvers.size(), -1);     // segment of each instance in the previous round
        int smax = 0;
        for (int r : g.members) smax = std::max(smax, b->solvers[r]->P.N);
        for (int s = 0; s < smax; ++s)
            for (int r : g.members) {
                const Params &P = b->solvers[r]->P;
                if (P.N <= s) continue;
                inst.push_back(r);
                step.push_back(P.N - 1 - s);
                dep.push_back(last[r]);
                last[r] = (int)inst.size() - 1;
                kofs.push_back(kofs.back() + P.K);
            }
        g.n_seg = (int)inst.size();
        g.flow_total = kofs.back();
        const size_t n = (size_t)g.n_seg;
        if ((e = cudaMalloc(&g.f_inst, sizeof(int) * n)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&g.f_step, sizeof(int) * n)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&g.f_dep, sizeof(int) * n)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&g.f_kofs, sizeof(long long) * (n + 1))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&g.f_done, sizeof(unsigned long long) * (n + 1))) != cudaSuccess) return e;
        if ((e = cudaMemcpy(g.f_inst, inst.data(), sizeof(int) * n, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(g.f_step, step.data(), sizeof(int) * n, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(g.f_dep, dep.data(), sizeof(int) * n, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(g.f_kofs, kofs.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_flow(srmc_batch *b, cudaStream_t st)
{
    cudaError_t e = build_flow(b);
    if (e != cudaSuccess) return e;
    if ((e = ensure_streams(b)) != cudaSuccess) return e;
    const int ng = (int)std::min(b->groups.size(), b->branch.size());
    if ((e = cudaEventRecord(b->ev[kBranchStreams], st)) != cudaSuccess) return e;
    for (int a = 0; a < ng; ++a)
        if ((e = cudaStreamWaitEvent(b->branch[a], b->ev[kBranchStreams], 0)) != cudaSuccess) return e;
    for (size_t q = 0; q < b->groups.size(); ++q) {
        const Group &g = b->groups[q];
        cudaStream_t x = b->branch[q % ng];
        if ((e = cudaMemsetAsync(g.f_done, 0, sizeof(unsigned long long) * (g.n_seg + 1), x)) != cudaSuccess)
            return e;
        srmc::FlowPlan F;
        F.params = b->d_params;
        F.inst = g.f_inst; F.step = g.f_step; F.kofs = g.f_kofs; F.dep = g.f_dep;
        F.done = g.f_done; F.next = g.f_done + g.n_seg; F.error = b->d_error;
        F.n_seg = g.n_seg; F.total = g.flow_total;
        const int occ = flow_occ_for(g.d)(g.lp1, g.mv, g.cv, g.threads);
        if (occ <= 0) return cudaErrorInvalidConfiguration;
        const int bps = (g.blocks_per_sm > 0 && g.blocks_per_sm < occ) ? g.blocks_per_sm : occ;
        long long grid = (long long)b->sms * bps;
        if (grid > g.flow_total) grid = g.flow_total;
        if ((e = flow_for(g.d)(F, g.lp1, g.mv, g.cv, (int)grid, g.threads, x)) != cudaSuccess) return e;
    }
    for (int a = 0; a < ng; ++a) {
        if ((e = cudaEventRecord(b->ev[a], b->branch[a])) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, b->ev[a], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_all(const srmc_batch *b, cudaStream_t st)
{
    int smax = 0;
    for (const auto &g : b->groups)
        for (const auto &r : g.rounds) smax = std::max(smax, r.s + 1);
    // round by round so that within a group round s+1 follows round s
    for (int s = 0; s < smax; ++s)
        for (const auto &g : b->groups)
            for (const auto &r : g.rounds)
                if (r.s == s) {
                    cudaError_t e = launch_round(b, g, r, g.threads, g.blocks_per_sm, st);
                    if (e != cudaSuccess) return e;
                }
    return cudaSuccess;
}

}  // namespace

namespace {
srmc_status ensure_graph(srmc_batch *b);
}

extern "C" {

srmc_status srmc_batch_create(srmc_solver *const *solvers, int n, srmc_batch **out)
{
    if (!out) return bfail(SRMC_ERR_INVALID_ARG, "srmc_batch_create: out is NULL");
    *out = nullptr;
    if (!solvers || n <= 0) return bfail(SRMC_ERR_INVALID_ARG, "srmc_batch_create: no solvers");
    int dev = 0;
    BATCH_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    for (int r = 0; r < n; ++r) {
        if (!solvers[r]) return bfail(SRMC_ERR_INVALID_ARG, "srmc_batch_create: NULL solver");
        if (solvers[r]->fp64) return bfail(SRMC_ERR_UNSUPPORTED, "srmc_batch_create: FP32 solvers only");
        if (solvers[r]->P.kind != 0)
            return bfail(SRMC_ERR_UNSUPPORTED, "srmc_batch_create: equal-size strata only");
        if (solvers[r]->exact || solvers[r]->dense)
            return bfail(SRMC_ERR_UNSUPPORTED, "srmc_batch_create: Euler dynamics with a diagonal sigma only");
        if (solvers[r]->lp2)
            return bfail(SRMC_ERR_UNSUPPORTED, "srmc_batch_create: LP0 and LP1 only");
        if (solvers[r]->P.model == srmc::MODEL_USER)
            return bfail(SRMC_ERR_UNSUPPORTED, "srmc_batch_create: built-in models only");
        if (solvers[r]->P.d > 8)
            return bfail(SRMC_ERR_UNSUPPORTED, "srmc_batch_create: d <= 8 only");
        if (solvers[r]->device != dev) return bfail(SRMC_ERR_INVALID_ARG, "srmc_batch_create: solver on another device");
    }
    srmc_batch *b = new srmc_batch();
    b->solvers.assign(solvers, solvers + n);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    // group by kernel variant
    for (int r = 0; r < n; ++r) {
        const srmc_solver *s = solvers[r];
        auto it = std::find_if(b->groups.begin(), b->groups.end(), [&](const Group &g) {
            return g.d == s->P.d && g.mv == srmc::kernel_mv(s) && g.lp1 == s->lp1 && g.cv == s->cv;
        });
        if (it == b->groups.end()) {
            Group g;
            g.d = s->P.d; g.mv = srmc::kernel_mv(s); g.lp1 = s->lp1; g.cv = s->cv;
            b->groups.push_back(g);
            it = b->groups.end() - 1;
        }
        it->members.push_back(r);
    }
    // rounds and their work lists
    std::vector<int> ints;
    std::vector<long long> kofs;
    for (auto &g : b->groups) {
        int smax = 0;
        for (int r : g.members) smax = std::max(smax, solvers[r]->P.N);
        for (int s = 0; s < smax; ++s) {
            Round rd;
            rd.s = s;
            rd.off = (long long)ints.size();
            rd.koff = (long long)kofs.size();
            std::vector<int> inst, step;
            long long acc = 0;
            kofs.push_back(0);
            for (int r : g.members) {
                const Params &P = solvers[r]->P;
                if (P.N > s) {
                    inst.push_back(r);
                    step.push_back(P.N - 1 - s);
                    acc += P.K;
                    kofs.push_back(acc);
                }
            }
            rd.n_active = (int)inst.size();
            rd.total = acc;
            ints.insert(ints.end(), inst.begin(), inst.end());
            ints.insert(ints.end(), step.begin(), step.end());
            g.rounds.push_back(rd);
        }
    }
    std::vector<Params> params(n);
    for (int r = 0; r < n; ++r) {
        params[r] = solvers[r]->P;
        const bool rows = solvers[r]->cv && !solvers[r]->cv_own;
        params[r].C16 = rows ? solvers[r]->C16 : nullptr;
        params[r].C64 = rows ? solvers[r]->C64 : nullptr;
        params[r].cv_own = solvers[r]->cv && solvers[r]->cv_own ? 1 : 0;
    }
    cudaError_t e = cudaMalloc(&b->d_params, sizeof(Params) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ints, sizeof(int) * std::max<size_t>(ints.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_kofs, sizeof(long long) * std::max<size_t>(kofs.size(), 1));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_params, params.data(), sizeof(Params) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !ints.empty())
        e = cudaMemcpy(b->d_ints, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !kofs.empty())
        e = cudaMemcpy(b->d_kofs, kofs.data(), sizeof(long long) * kofs.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        batch_free(b);
        delete b;
        return bfail(e == cudaErrorMemoryAllocation ? SRMC_ERR_OOM : SRMC_ERR_CUDA,
                     std::string("srmc_batch_create: ") + cudaGetErrorString(e));
    }
    *out = b;
    return SRMC_OK;
}

void srmc_batch_destroy(srmc_batch *b)
{
    if (!b) return;
    batch_free(b);
    delete b;
}

srmc_status srmc_batch_tune(srmc_batch *b, void *stream, int *out_threads, int max_out, int *n_groups)
{
    if (!b) return bfail(SRMC_ERR_INVALID_ARG, "srmc_batch_tune: NULL batch");
    b->mode = MODE_ROUNDS;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    BATCH_CUDA(cudaEventCreate(&e0), "event");
    BATCH_CUDA(cudaEventCreate(&e1), "event");
    const int cand_threads[3] = {64, 128, 256};
    for (auto &g : b->groups) {
        // time the first rounds (all instances active; short paths) and one
        // middle round (long paths) for every candidate, twice, keep the best
        std::vector<const Round *> probe;
        for (const auto &r : g.rounds)
            if (r.s < 2) probe.push_back(&r);
        if (!g.rounds.empty()) probe.push_back(&g.rounds[g.rounds.size() / 2]);
        float best = 1e30f;
        int best_t = 256, best_b = 0;
        for (int t : cand_threads) {
            const int occ = occ_for(g.d)(false, g.lp1, g.mv, g.cv, t);
            if (occ <= 0) continue;
            const int cand_b[3] = {occ, std::max(1, occ / 2), std::max(1, occ * 2 / 3)};
            for (int bps : cand_b) {
                float tot = 0.0f;
                for (int rep = 0; rep < 2; ++rep) {
                    BATCH_CUDA(cudaEventRecord(e0, st), "event record");
                    for (const Round *r : probe) BATCH_CUDA(launch_round(b, g, *r, t, bps, st), "tune launch");
                    BATCH_CUDA(cudaEventRecord(e1, st), "event record");
                    BATCH_CUDA(cudaEventSynchronize(e1), "event sync");
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep == 1) tot = ms;
                }
                if (tot < best) { best = tot; best_t = t; best_b = bps; }
            }
        }
        g.threads = best_t;
        g.blocks_per_sm = best_b;
    }
    // Both strategies with the chosen block sizes (BRANCHES: every solver of a
    // group takes the group's threads), one warm-up and one timed pass each.
    for (auto &g : b->groups)
        for (int r : g.members) {
            srmc_solver *s = b->solvers[r];
            if (s->threads != g.threads) {
                s->threads = g.threads;
                if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
            }
        }
    float tm[3] = {0.0f, 0.0f, 0.0f};
    for (int mode = 0; mode < 3; ++mode) {
        b->mode = mode;
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        srmc_status ss = ensure_graph(b);          // capture outside the timed pass
        if (ss != SRMC_OK) return ss;
        BATCH_CUDA(cudaEventRecord(e0, st), "event record");
        BATCH_CUDA(cudaGraphLaunch(b->graph, st), "batch graph launch");
        BATCH_CUDA(cudaEventRecord(e1, st), "event record");
        BATCH_CUDA(cudaEventSynchronize(e1), "event sync");
        cudaEventElapsedTime(&tm[mode], e0, e1);
    }
    b->mode = MODE_ROUNDS;
    for (int mode = 1; mode < 3; ++mode)
        if (tm[mode] < tm[b->mode]) b->mode = mode;
    for (int mode = 0; mode < 3; ++mode) b->strategy_ms[mode] = tm[mode];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    if (n_groups) *n_groups = (int)b->groups.size();
    if (out_threads)
        for (int a = 0; a < (int)b->groups.size() && a < max_out; ++a) out_threads[a] = b->groups[a].threads;
    return SRMC_OK;
}

int srmc_batch_mode(const srmc_batch *b) { return b ? b->mode : -1; }

srmc_status srmc_batch_strategy_ms(const srmc_batch *b, float out_ms[3])
{
    if (!b || !out_ms) return bfail(SRMC_ERR_INVALID_ARG, "srmc_batch_strategy_ms: NULL argument");
    for (int a = 0; a < 3; ++a) out_ms[a] = b->strategy_ms[a];
    return SRMC_OK;
}

srmc_status srmc_batch_stats(srmc_batch *b, unsigned long long *timeouts)
{
    if (!b || !timeouts) return bfail(SRMC_ERR_INVALID_ARG, "srmc_batch_stats: NULL argument");
    unsigned e = 0;
    BATCH_CUDA(cudaDeviceSynchronize(), "srmc_batch_stats: synchronize");
    if (b->d_error) BATCH_CUDA(cudaMemcpy(&e, b->d_error, sizeof(unsigned), cudaMemcpyDeviceToHost), "srmc_batch_stats");
    *timeouts = e;
    return SRMC_OK;
}

srmc_status srmc_batch_set_mode(srmc_batch *b, int mode)
{
    if (!b || (mode != MODE_ROUNDS && mode != MODE_BRANCHES && mode != MODE_FLOW))
        return bfail(SRMC_ERR_INVALID_ARG, "srmc_batch_set_mode: bad argument");
    if (b->mode != mode && b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    b->mode = mode;
    return SRMC_OK;
}

srmc_status srmc_batch_solve(srmc_batch *b, void *stream)
{
    if (!b) return bfail(SRMC_ERR_INVALID_ARG, "srmc_batch_solve: NULL batch");
    srmc_status ss = ensure_graph(b);
    if (ss != SRMC_OK) return ss;
    BATCH_CUDA(cudaGraphLaunch(b->graph, (cudaStream_t)stream), "batch graph launch");
    for (srmc_solver *s : b->solvers) s->done_from = 0;
    return SRMC_OK;
}

}  // extern "C"

namespace {
// Capture the strategy's launches into b->graph if it is not there yet.
srmc_status ensure_graph(srmc_batch *b)
{
    if (!b->graph) {
        if (!b->cap_stream)
            BATCH_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "graph stream");
        // allocations and copies of the FLOW plan happen before the capture
        if (b->mode != MODE_ROUNDS) BATCH_CUDA(ensure_streams(b), "batch streams");
        if (b->mode == MODE_FLOW) BATCH_CUDA(build_flow(b), "batch flow plan");
        cudaGraph_t g = nullptr;
        BATCH_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t le = b->mode == MODE_ROUNDS ? enqueue_all(b, b->cap_stream)
                         : b->mode == MODE_BRANCHES ? enqueue_branches(b, b->cap_stream)
                                                    : enqueue_flow(b, b->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &g);
        if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return bfail(SRMC_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(le)); }
        if (ce != cudaSuccess) return bfail(SRMC_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(ce));
        cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) { b->graph = nullptr; return bfail(SRMC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie)); }
    }
    return SRMC_OK;
}
}  // namespace
