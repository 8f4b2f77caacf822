// sg_sched.cu -- the native core of continuous batching (include/sg_sched.h).
//
// Host code only: the kernels are the batch steps of sg_batch.cu, called
// through the public C ABI (sg_batch_ca_plan_host, sg_batch_ca_steps).  An
// iteration walks the gaskets that hold requests, advances each resident one
// by min(fuse, steps left in its head request), groups them by the halo that
// advance needs (1 step; 2..4; 5..8; 9..16), writes every group's
// work list into one page-locked image, copies it to the device in one
// asynchronous copy and issues one batched launch per group.  The host-side
// state (queues, which buffer is current) is updated as the work is
// enqueued: stream order makes it true by the time the device gets there.
//
// Two image slots alternate between iterations.  Before a slot is rewritten
// the host waits for the event recorded after the copy that last read it,
// which normally completed long before (it belongs to the iteration before
// the previous one).
#include <algorithm>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "sg.h"
#include "sg_internal.h"
#include "sg_sched.h"

namespace {

constexpr int kSlots = 2;
constexpr int kMaxCount = 65535;

struct Request {
    int64_t id;
    int32_t steps;
    int32_t left;
};

struct Gasket {
    int32_t level = 0;
    uint64_t cells = 0;            // 3^level
    uint8_t *cur = nullptr, *nxt = nullptr;
    std::deque<Request> queue;
    uint64_t last_use = 0, steps_done = 0;
    bool pending = false;          // listed in sg_sched::pending (has queued requests)
    bool inject = false;           // fail the next launch that holds it
};

uint64_t pow3(int e)
{
    uint64_t v = 1;
    while (e-- > 0) v *= 3;
    return v;
}

uint64_t up16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }

}  // namespace

struct sg_sched {
    int count = 0, rho = 0, fuse = 1, s = 0;
    sg_launch_opts opts{};
    bool have_opts = false;
    std::vector<Gasket> g;
    std::vector<int32_t> pending;                  // gaskets with queued requests
    int classes = 1;                               // halo classes in use (by fuse)
    uint64_t slot_bytes = 0;
    unsigned char *img[kSlots] = {nullptr, nullptr};   // page-locked images
    void *dev[kSlots] = {nullptr, nullptr};            // device work lists
    cudaEvent_t copied[kSlots] = {nullptr, nullptr};
    bool in_use[kSlots] = {false, false};
    int slot = 0;
    uint64_t iteration = 0;
    // per-iteration scratch, kept to avoid allocations
    std::vector<int32_t> still;
    std::vector<std::vector<int32_t>> members;
    std::vector<sg_batch_plan> plans;
    std::vector<sg_status> planned;
    std::vector<int> lv, kk;
    std::vector<int> adv;                          // per gasket: this iteration's advance
    std::vector<uint8_t *> pa, pb;
};

namespace {

sg_status cuda_err(cudaError_t e) { return sg::set_last_cuda_error(e); }

void free_sched(sg_sched *s)
{
    for (int j = 0; j < kSlots; ++j) {
        if (s->copied[j]) {
            cudaEventSynchronize(s->copied[j]);
            cudaEventDestroy(s->copied[j]);
        }
        if (s->img[j]) cudaFreeHost(s->img[j]);
        if (s->dev[j]) cudaFree(s->dev[j]);
    }
    delete s;
}

// The launch class of an advance of k steps: the halo its fused launch
// stages (sg_batch_ca_steps sizes it from the launch's k) -- 1 step (the
// single-step kernel), 2..4, 5..8, 9..16.
constexpr int kClasses = 4;
int class_of(int k) { return k <= 1 ? 0 : k <= 4 ? 1 : k <= 8 ? 2 : 3; }

}  // namespace

extern "C" {

sg_status sg_sched_create(int count, const int *levels, int rho, int fuse,
                          const sg_launch_opts *opts, sg_sched **out)
{
    if (out == nullptr || levels == nullptr || count < 1 || count > kMaxCount) return SG_EINVAL;
    *out = nullptr;
    if (rho != 16 && rho != 32 && rho != 64) return SG_EUNSUPPORTED;
    if (fuse < 1 || fuse > SG_FUSE_MAX) return SG_EINVAL;
    int s = 0;
    while ((1 << s) < rho) ++s;
    for (int i = 0; i < count; ++i)
        if (levels[i] < s || levels[i] > 16) return SG_EINVAL;
    sg::LaunchCfg probe;
    if (opts != nullptr && !sg::read_launch_opts(opts, &probe)) return SG_EINVAL;
    sg_sched *S = new (std::nothrow) sg_sched;
    if (S == nullptr) return SG_ECUDA;
    S->count = count;
    S->rho = rho;
    S->fuse = fuse;
    S->s = s;
    if (opts != nullptr) {
        S->opts = *opts;
        S->have_opts = true;
    }
    S->g.resize(count);
    for (int i = 0; i < count; ++i) {
        S->g[i].level = levels[i];
        S->g[i].cells = pow3(levels[i]);
    }
    S->classes = class_of(fuse) + 1;
    S->members.resize(kClasses);
    S->plans.resize(kClasses);
    S->planned.resize(kClasses);
    S->adv.assign(count, 0);
    // every group's work list at a 16-byte boundary: the whole batch's
    // layout plus 64 bytes of slack for each group's own layout and alignment
    S->slot_bytes = up16(sg_batch_workspace_bytes(count) + 64ull * kClasses + 64);
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < kSlots && e == cudaSuccess; ++j) {
        e = cudaHostAlloc(reinterpret_cast<void **>(&S->img[j]), S->slot_bytes,
                          cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&S->dev[j], S->slot_bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->copied[j], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        free_sched(S);
        return cuda_err(e);
    }
    *out = S;
    return SG_OK;
}

sg_status sg_sched_destroy(sg_sched *s)
{
    if (s == nullptr) return SG_EINVAL;
    free_sched(s);
    return SG_OK;
}

sg_status sg_sched_set_buffers(sg_sched *s, int g, uint8_t *cur, uint8_t *nxt)
{
    if (s == nullptr || g < 0 || g >= s->count) return SG_EINVAL;
    if ((cur == nullptr) != (nxt == nullptr)) return SG_EINVAL;
    if (cur != nullptr &&
        (cur == nxt || ((uintptr_t)cur & 15) != 0 || ((uintptr_t)nxt & 15) != 0))
        return SG_EINVAL;
    s->g[g].cur = cur;
    s->g[g].nxt = nxt;
    return SG_OK;
}

sg_status sg_sched_submit(sg_sched *s, int n, const int32_t *gasket, const int64_t *request,
                          const int32_t *steps)
{
    if (s == nullptr || n < 0) return SG_EINVAL;
    if (n == 0) return SG_OK;
    if (gasket == nullptr || request == nullptr || steps == nullptr) return SG_EINVAL;
    for (int i = 0; i < n; ++i)
        if (gasket[i] < 0 || gasket[i] >= s->count || steps[i] < 1) return SG_EINVAL;
    for (int i = 0; i < n; ++i) {
        Gasket &G = s->g[gasket[i]];
        G.queue.push_back(Request{request[i], steps[i], steps[i]});
        if (!G.pending) {
            G.pending = true;
            s->pending.push_back(gasket[i]);
        }
    }
    return SG_OK;
}

sg_status sg_sched_waiting(const sg_sched *s, int32_t *out, int max, int *n)
{
    if (s == nullptr || n == nullptr || max < 0 || (max > 0 && out == nullptr)) return SG_EINVAL;
    int w = 0;
    for (int32_t g : s->pending)
        if (s->g[g].cur == nullptr && !s->g[g].queue.empty() && w < max) out[w++] = g;
    *n = w;
    return SG_OK;
}

sg_status sg_sched_gasket(const sg_sched *s, int g, sg_sched_gasket_info *info)
{
    if (s == nullptr || info == nullptr || g < 0 || g >= s->count) return SG_EINVAL;
    const Gasket &G = s->g[g];
    *info = sg_sched_gasket_info{};
    info->level = G.level;
    info->queued = (int32_t)G.queue.size();
    info->head_left = G.queue.empty() ? 0 : G.queue.front().left;
    info->resident = G.cur != nullptr;
    info->cur = (uint64_t)(uintptr_t)G.cur;
    info->nxt = (uint64_t)(uintptr_t)G.nxt;
    info->last_use = G.last_use;
    info->steps_done = G.steps_done;
    return SG_OK;
}

sg_status sg_sched_drop(sg_sched *s, int g, int64_t *request, int32_t *steps_run, int max,
                        int *n)
{
    if (s == nullptr || n == nullptr || g < 0 || g >= s->count) return SG_EINVAL;
    Gasket &G = s->g[g];
    if ((int64_t)G.queue.size() > (int64_t)max || (max > 0 && (!request || !steps_run)))
        return SG_EINVAL;
    int w = 0;
    for (const Request &q : G.queue) {
        request[w] = q.id;
        steps_run[w] = q.steps - q.left;
        ++w;
    }
    G.queue.clear();
    *n = w;
    return SG_OK;          // g leaves the pending list at the next iteration
}

sg_status sg_sched_inject_launch_failure(sg_sched *s, int g)
{
    if (s == nullptr || g < 0 || g >= s->count) return SG_EINVAL;
    s->g[g].inject = true;
    return SG_OK;
}

sg_status sg_sched_step(sg_sched *s, void *stream, sg_sched_result *res)
{
    if (s == nullptr || res == nullptr) return SG_EINVAL;
    res->n_completed = res->n_failed = res->active = res->launches = 0;
    res->cell_steps = 0;
    res->iteration = 0;
    // every gasket may complete or fail one request per iteration
    int tried = 0;
    for (int32_t g : s->pending)
        if (s->g[g].cur != nullptr && !s->g[g].queue.empty()) ++tried;
    if (tried == 0) {
        // drop gaskets whose queues were emptied (sg_sched_drop)
        s->still.clear();
        for (int32_t g : s->pending) {
            if (s->g[g].queue.empty()) s->g[g].pending = false;
            else s->still.push_back(g);
        }
        s->pending.swap(s->still);
        return SG_OK;
    }
    if (res->max_entries < tried || res->completed == nullptr ||
        res->completed_gasket == nullptr || res->failed == nullptr ||
        res->failed_gasket == nullptr || res->failed_steps_run == nullptr)
        return SG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;

    // the resident gaskets with requests: each advances by min(fuse, steps
    // left in its head request), grouped by the halo class of that advance
    for (auto &m : s->members) m.clear();
    for (int32_t g : s->pending) {
        Gasket &G = s->g[g];
        if (G.cur == nullptr || G.queue.empty()) continue;
        const int k = std::min(s->fuse, G.queue.front().left);
        s->adv[g] = k;
        s->members[class_of(k)].push_back(g);
    }

    // the image slot: wait for the copy that last read it
    const int j = s->slot;
    if (s->in_use[j]) {
        const cudaError_t e = cudaEventSynchronize(s->copied[j]);
        if (e != cudaSuccess) return cuda_err(e);
    }
    const uint64_t iter = ++s->iteration;
    res->iteration = iter;
    auto &plans = s->plans;
    auto &planned = s->planned;
    std::fill(planned.begin(), planned.end(), SG_EINVAL);
    uint64_t off = 0;
    int launch_k[kClasses] = {1, 1, 1, 1};
    for (int gi = 0; gi < s->classes; ++gi) {
        const auto &m = s->members[gi];
        if (m.empty()) continue;
        const int cnt = (int)m.size();
        s->lv.resize(cnt);
        s->kk.resize(cnt);
        s->pa.resize(cnt);
        s->pb.resize(cnt);
        for (int i = 0; i < cnt; ++i) {
            const Gasket &G = s->g[m[i]];
            s->lv[i] = G.level;
            s->kk[i] = s->adv[m[i]];
            launch_k[gi] = std::max(launch_k[gi], s->kk[i]);
            s->pa[i] = G.cur;
            s->pb[i] = G.nxt;
        }
        const uint64_t need = sg_batch_workspace_bytes(cnt);
        // single steps need no per-gasket counts; the fused classes carry them
        planned[gi] = sg_batch_ca_plan_host(cnt, s->lv.data(), gi == 0 ? nullptr : s->kk.data(),
                                            s->pa.data(), s->pb.data(), s->rho, s->img[j] + off,
                                            need, static_cast<unsigned char *>(s->dev[j]) + off,
                                            need, &plans[gi]);
        if (planned[gi] == SG_OK) off = up16(off + need);
    }
    if (off > 0) {
        cudaError_t e = cudaMemcpyAsync(s->dev[j], s->img[j], off, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaEventRecord(s->copied[j], st);
        if (e != cudaSuccess) return cuda_err(e);
        s->in_use[j] = true;
        s->slot = (j + 1) % kSlots;
    }

    // one launch per group; the host state follows the enqueued work
    const sg_launch_opts *opts = s->have_opts ? &s->opts : nullptr;
    for (int gi = 0; gi < s->classes; ++gi) {
        const auto &m = s->members[gi];
        if (m.empty()) continue;
        const int k = launch_k[gi];
        sg_status st_launch = planned[gi];
        bool injected = false;
        for (int32_t g : m)
            if (s->g[g].inject) injected = true;
        if (st_launch == SG_OK && injected) {
            st_launch = SG_ECUDA;
            sg::set_last_error_message("sg_sched_step: injected launch failure");
            for (int32_t g : m) s->g[g].inject = false;
        } else if (st_launch == SG_OK) {
            st_launch = sg_batch_ca_steps(&plans[gi], 0, k, opts, stream);
            if (st_launch == SG_OK) ++res->launches;
        }
        res->active += (int32_t)m.size();
        for (int32_t g : m) {
            Gasket &G = s->g[g];
            G.last_use = iter;
            Request &h = G.queue.front();
            if (st_launch != SG_OK) {            // nothing ran: the head request fails
                res->failed[res->n_failed] = h.id;
                res->failed_gasket[res->n_failed] = g;
                res->failed_steps_run[res->n_failed] = h.steps - h.left;
                ++res->n_failed;
                G.queue.pop_front();
                continue;
            }
            const int a = s->adv[g];             // this gasket's own advance (<= k)
            std::swap(G.cur, G.nxt);
            G.steps_done += (uint64_t)a;
            res->cell_steps += G.cells * (uint64_t)a;
            h.left -= a;
            if (h.left == 0) {
                res->completed[res->n_completed] = h.id;
                res->completed_gasket[res->n_completed] = g;
                ++res->n_completed;
                G.queue.pop_front();
            }
        }
    }
    // keep the gaskets that still hold requests
    s->still.clear();
    for (int32_t g : s->pending) {
        if (s->g[g].queue.empty()) s->g[g].pending = false;
        else s->still.push_back(g);
    }
    s->pending.swap(s->still);
    return SG_OK;
}

}  // extern "C"
