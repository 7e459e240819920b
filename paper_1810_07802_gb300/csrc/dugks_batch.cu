// dugks_batch.cu -- batches of independent solvers advanced together.
//
// Members are grouped by kernel variant (precision x model x y-boundary x
// tile shape x reconstruction).
// Each group owns a device array of per-problem descriptors (buffers,
// constants, tensor maps, step counter), a work list of (problem, tile)
// items and 1 + members counters.  By default K steps of a group are one
// persistent launch (a queue of K x items taken in step order; a tile waits
// only for its own member's previous step, counted per member) plus a tiny
// launch that advances every member's buffer parity and step count; the
// other mode launches one grid per step.  The launches of K steps are
// captured once into a CUDA graph and replayed until membership changes (one
// graph of 16 steps and one of a single step).
//
// A member of at least kSoloTiles tiles fills the GPU by itself for several
// waves: it is stepped by the single-problem kernel (as by dugks_step), whose
// constants are parameter-bank operands of the arithmetic rather than loads
// from its descriptor (about 10 % faster on a 2048^2 grid), and the launch
// cost is hidden behind its run time.  Which path a member takes depends on
// its own size only, so a member's result does not depend on what else is in
// the batch.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "dugks.h"
#include "dugks_internal.h"
#include "dugks_trace.h"

using dugks::InstDesc;
using dugks::fill_desc;

namespace {

constexpr int kMaxTiles = 4;   // compiled tile shapes per precision, at most
constexpr long long kSoloTiles = 2048;   // about 4.5 waves of 3 CTAs on each of 152 SMs

long long member_tiles(const dugks_ctx *c) {
    const int tx = c->fp32 ? dugks::tile_dim<float>(c->tile, 0) : dugks::tile_dim<double>(c->tile, 0);
    const int ty = c->fp32 ? dugks::tile_dim<float>(c->tile, 1) : dugks::tile_dim<double>(c->tile, 1);
    return (long long)((c->P.nx + tx - 1) / tx) * ((c->P.ny + ty - 1) / ty);
}

struct Group {
    bool fp32 = false, coupled = false, wally = false, upw = false;
    int tile = 0;
    std::vector<dugks_ctx *> members;
    std::vector<unsigned char> h_desc;   // host image of the descriptor array
    std::vector<int2> h_work;
    void *d_desc = nullptr;
    int2 *d_work = nullptr;
    unsigned *d_ctr = nullptr;           // queue head + one step counter per member
    size_t desc_cap = 0, work_cap = 0, ctr_cap = 0;   // bytes / items / counters allocated
    int nwork = 0;
};

size_t desc_size(bool fp32) { return fp32 ? sizeof(InstDesc<float>) : sizeof(InstDesc<double>); }

dugks_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return DUGKS_OK;
    return e == cudaErrorMemoryAllocation ? DUGKS_ERR_OOM : DUGKS_ERR_CUDA;
}

}  // namespace

struct dugks_batch_ctx {
    cudaStream_t st = nullptr;
    std::vector<dugks_ctx *> members;
    std::vector<dugks_ctx *> solo;   // members stepped by the single-problem kernel
    bool grouped = false;            // some group is non-empty
    static constexpr int kGroups = 16 * kMaxTiles;
    Group groups[kGroups];   // index: (upw * 8 + fp32 * 4 + coupled * 2 + wally) * kMaxTiles + tile
    bool dirty = true;
    bool persistent = false;         // K steps per launch (else one grid launch per step)
    // CUDA graphs of one step and of kUnroll steps of the current membership
    static constexpr int kUnroll = 16;
    cudaGraphExec_t exec = nullptr, exec_k = nullptr;

    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (exec_k) cudaGraphExecDestroy(exec_k);
        exec = exec_k = nullptr;
    }

    // Rebuilds the host images (descriptors always, work lists when dirty) and uploads them.
    cudaError_t upload() {
        if (dirty) {
            solo.clear();
            for (dugks_ctx *c : members)
                if (member_tiles(c) >= kSoloTiles) solo.push_back(c);
            grouped = false;
        }
        for (int gi = 0; gi < kGroups; gi++) {
            Group &g = groups[gi];
            if (dirty) {
                const int v = gi / kMaxTiles;
                g.upw = v & 8;
                g.fp32 = v & 4;
                g.coupled = v & 2;
                g.wally = v & 1;
                g.tile = gi % kMaxTiles;
                g.members.clear();
                for (dugks_ctx *c : members)
                    if (c->fp32 == g.fp32 && c->coupled == g.coupled && c->wally == g.wally && c->tile == g.tile &&
                        c->upw == g.upw && member_tiles(c) < kSoloTiles)
                        g.members.push_back(c);
                grouped = grouped || !g.members.empty();
                const int tx = g.fp32 ? dugks::tile_dim<float>(g.tile, 0) : dugks::tile_dim<double>(g.tile, 0);
                const int ty = g.fp32 ? dugks::tile_dim<float>(g.tile, 1) : dugks::tile_dim<double>(g.tile, 1);
                g.h_work.clear();
                for (size_t i = 0; i < g.members.size(); i++) {
                    const dugks_ctx *c = g.members[i];
                    const int n = ((c->P.nx + tx - 1) / tx) * ((c->P.ny + ty - 1) / ty);
                    for (int t = 0; t < n; t++) g.h_work.push_back(make_int2((int)i, t));
                }
                g.nwork = (int)g.h_work.size();
            }
            if (g.members.empty()) continue;
            const size_t ds = desc_size(g.fp32);
            g.h_desc.assign(ds * g.members.size(), 0);
            const int tx = g.fp32 ? dugks::tile_dim<float>(g.tile, 0) : dugks::tile_dim<double>(g.tile, 0);
            const int ty = g.fp32 ? dugks::tile_dim<float>(g.tile, 1) : dugks::tile_dim<double>(g.tile, 1);
            for (size_t i = 0; i < g.members.size(); i++) {
                const dugks_ctx *c = g.members[i];
                if (g.fp32)
                    fill_desc(reinterpret_cast<InstDesc<float> *>(g.h_desc.data()) + i, c, c->phf, tx, ty);
                else
                    fill_desc(reinterpret_cast<InstDesc<double> *>(g.h_desc.data()) + i, c, c->phd, tx, ty);
            }
            // grow the device arrays (capacity doubling; the graph holds their addresses)
            if (g.h_desc.size() > g.desc_cap) {
                drop_graph();
                if (g.d_desc) cudaFree(g.d_desc);
                g.desc_cap = std::max(g.h_desc.size(), 2 * g.desc_cap);
                cudaError_t e = cudaMalloc(&g.d_desc, g.desc_cap);
                if (e != cudaSuccess) { g.d_desc = nullptr; g.desc_cap = 0; return e; }
            }
            if (g.h_work.size() > g.work_cap) {
                drop_graph();
                if (g.d_work) cudaFree(g.d_work);
                g.work_cap = std::max(g.h_work.size(), 2 * g.work_cap);
                cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&g.d_work), g.work_cap * sizeof(int2));
                if (e != cudaSuccess) { g.d_work = nullptr; g.work_cap = 0; return e; }
            }
            if (1 + g.members.size() > g.ctr_cap) {
                drop_graph();
                if (g.d_ctr) cudaFree(g.d_ctr);
                g.ctr_cap = std::max(1 + g.members.size(), 2 * g.ctr_cap);
                cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&g.d_ctr), g.ctr_cap * sizeof(unsigned));
                if (e != cudaSuccess) { g.d_ctr = nullptr; g.ctr_cap = 0; return e; }
            }
            cudaError_t e = cudaMemcpyAsync(g.d_desc, g.h_desc.data(), g.h_desc.size(), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess && dirty)
                e = cudaMemcpyAsync(g.d_work, g.h_work.data(), g.h_work.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return e;
        }
        if (dirty) drop_graph();
        dirty = false;
        return cudaSuccess;
    }

    // k batched steps: every non-empty group's launches and descriptor advances.
    cudaError_t enqueue_steps(int k) {
        for (Group &g : groups) {
            if (g.members.empty()) continue;
            unsigned *ctr = persistent ? g.d_ctr : nullptr;
            cudaError_t e = g.fp32 ? dugks::launch_batch_step<float>(g.tile, g.upw, static_cast<InstDesc<float> *>(g.d_desc),
                                                                     g.d_work, g.nwork, (int)g.members.size(),
                                                                     g.coupled, g.wally, k, ctr, st)
                                   : dugks::launch_batch_step<double>(g.tile, g.upw, static_cast<InstDesc<double> *>(g.d_desc),
                                                                      g.d_work, g.nwork, (int)g.members.size(),
                                                                      g.coupled, g.wally, k, ctr, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }

    // Captures `steps` consecutive batched steps into one executable graph.
    cudaError_t capture(int steps, cudaGraphExec_t *out) {
        for (Group &g : groups) {
            if (g.members.empty()) continue;
            cudaError_t e = g.fp32 ? dugks::batch_prepare<float>(g.tile, g.coupled, g.wally, g.upw)
                                   : dugks::batch_prepare<double>(g.tile, g.coupled, g.wally, g.upw);
            if (e != cudaSuccess) return e;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t el = enqueue_steps(steps);
        e = cudaStreamEndCapture(st, &graph);
        if (el != cudaSuccess) e = el;
        if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) *out = nullptr;
        return e;
    }
};

extern "C" {

dugks_status dugks_batch_create(void *cuda_stream, dugks_batch *out) {
    if (!out) return DUGKS_ERR_ARG;
    *out = nullptr;
    dugks_batch_ctx *b = new (std::nothrow) dugks_batch_ctx();
    if (!b) return DUGKS_ERR_OOM;
    b->st = static_cast<cudaStream_t>(cuda_stream);
    *out = b;
    return DUGKS_OK;
}

dugks_status dugks_batch_add(dugks_batch b, dugks_handle h) {
    if (!b || !h) return DUGKS_ERR_ARG;
    if (std::find(b->members.begin(), b->members.end(), h) != b->members.end()) return DUGKS_ERR_ARG;
    b->members.push_back(h);
    b->dirty = true;
    return DUGKS_OK;
}

dugks_status dugks_batch_remove(dugks_batch b, dugks_handle h) {
    if (!b || !h) return DUGKS_ERR_ARG;
    auto it = std::find(b->members.begin(), b->members.end(), h);
    if (it == b->members.end()) return DUGKS_ERR_ARG;
    b->members.erase(it);
    b->dirty = true;
    return DUGKS_OK;
}

int32_t dugks_batch_size(dugks_batch b) { return b ? (int32_t)b->members.size() : -1; }

dugks_status dugks_batch_step(dugks_batch b, int64_t nsteps) {
    dugks::TraceRange trace_("dugks_batch_step");
    if (!b || nsteps < 0) return DUGKS_ERR_ARG;
    if (nsteps == 0 || b->members.empty()) return DUGKS_OK;
    cudaError_t e = b->upload();
    // whole blocks of kUnroll steps as one graph launch each, the rest one step per launch
    const int64_t blocks = nsteps / dugks_batch_ctx::kUnroll, rest = nsteps % dugks_batch_ctx::kUnroll;
    if (e == cudaSuccess && b->grouped) {
        if (blocks > 0 && !b->exec_k) e = b->capture(dugks_batch_ctx::kUnroll, &b->exec_k);
        if (e == cudaSuccess && rest > 0 && !b->exec) e = b->capture(1, &b->exec);
        for (int64_t n = 0; n < blocks && e == cudaSuccess; n++) e = cudaGraphLaunch(b->exec_k, b->st);
        for (int64_t n = 0; n < rest && e == cudaSuccess; n++) e = cudaGraphLaunch(b->exec, b->st);
    }
    if (e != cudaSuccess) return from_cuda(e);
    for (Group &g : b->groups)
        for (dugks_ctx *c : g.members) {
            c->steps += nsteps;
            c->cur ^= (int)(nsteps & 1);
        }
    // large members: their own launches, on the batch's stream, in member order
    for (dugks_ctx *c : b->solo) {
        e = dugks::step_on(c, nsteps, b->st);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return DUGKS_OK;
}

dugks_status dugks_batch_set_persistent(dugks_batch b, int32_t on) {
    if (!b) return DUGKS_ERR_ARG;
    if (b->persistent != (on != 0)) {
        cudaError_t e = cudaStreamSynchronize(b->st);   // graphs in flight finish before they are dropped
        b->persistent = on != 0;
        b->drop_graph();
        if (e != cudaSuccess) return from_cuda(e);
    }
    return DUGKS_OK;
}

dugks_status dugks_batch_sync(dugks_batch b) {
    dugks::TraceRange trace_("dugks_batch_sync");
    if (!b) return DUGKS_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return from_cuda(e);
    dugks_status worst = DUGKS_OK;
    for (dugks_ctx *c : b->members) {
        dugks_status s = dugks_sync(c);
        if (s != DUGKS_OK && worst == DUGKS_OK) worst = s;
    }
    return worst;
}

dugks_status dugks_batch_destroy(dugks_batch b) {
    if (!b) return DUGKS_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(b->st);
    b->drop_graph();
    for (Group &g : b->groups) {
        if (g.d_desc) cudaFree(g.d_desc);
        if (g.d_work) cudaFree(g.d_work);
        if (g.d_ctr) cudaFree(g.d_ctr);
    }
    delete b;
    return from_cuda(e);
}

}  // extern "C"
