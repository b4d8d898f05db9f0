// batch.cu -- many independent lattices advanced by one persistent launch
// per time step (the extern "C" pflbm_batch_* entry points of pflbm.h).
//
// A batch holds, in device memory, one step descriptor per lattice for each
// parity of the ping-pong state (set 0: in = current copy, out = the other;
// set 1: swapped). A step is, by schedule kernel: 1, one launch of
// k_step_batch over a work list of (lattice, first tile) items; 2, one launch
// of the staged kernel over its work list; 3 (the default for FP32 and 16-bit
// storage), one launch of the two-node kernel per group of lattices of one
// size and viscosity mode, its descriptors passed in the launch's parameters
// (grid = tiles x lattices), the groups' launches forked onto side streams and
// joined back. With use_graph the launches of PFLBM_BATCH_GRAPH_STEPS steps
// are captured once in a CUDA graph and replayed; in it each group takes its
// steps back to back on its stream, and the streams join once per replay.
#include <algorithm>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "pflbm_internal.cuh"

namespace pfk {
int set_error(int code, const char* msg);
int materialize_handle(pflbm_t* h);
int post_status(pflbm_t* h);
}  // namespace pfk

using namespace pfk;

struct pflbm_batch {
    int precision = PFLBM_FP32;
    int device = 0;
    cudaStream_t stream = nullptr;
    pflbm_schedule_t sched{};
    std::vector<pflbm_t*> hs;
    std::vector<int> cur0;        // each lattice's state copy when descriptors were written
    int phase = 0;                // steps taken since then, mod 2
    size_t args_bytes = 0;
    int cap_lattices = 0, cap_work = 0;
    void* d_args[2] = {nullptr, nullptr};
    bool staged = false;          // staged (TMA ring) kernel, int4 items; else int2 items
    bool by_class = false;        // two-node kernel, one launch per group of same-size lattices
    struct ClassLaunch {
        int vv, nx, ny, count;
        std::vector<unsigned char> descs[2];   // count step descriptors of each set (host)
    };
    std::vector<ClassLaunch> classes;
    // per-class launches run side by side: forked from the batch's stream to
    // these streams and joined back (in the captured graph as well)
    static constexpr int kForks = 4;
    cudaStream_t fork_stream[kForks] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kForks] = {};
    void* d_work = nullptr;
    int n_work = 0;
    int grid = 0;
    long long nodes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_n_work = -1;
    void* (*alloc_fn)(size_t, void*) = nullptr;
    void (*free_fn)(void*, size_t, void*) = nullptr;
    void* alloc_ctx = nullptr;
};

namespace {

int balloc(pflbm_batch_t* b, void** p, size_t bytes)
{
    *p = nullptr;
    if (b->alloc_fn) {
        *p = b->alloc_fn(bytes, b->alloc_ctx);
        return *p ? PFLBM_OK : set_error(PFLBM_ENOMEM, "batch: allocator callback returned NULL");
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(PFLBM_ENOMEM, "batch: cudaMalloc failed");
    }
    return PFLBM_OK;
}

void bfree(pflbm_batch_t* b, void* p, size_t bytes)
{
    if (!p) return;
    if (b->free_fn)
        b->free_fn(p, bytes, b->alloc_ctx);
    else
        cudaFree(p);
}

void drop_graph(pflbm_batch_t* b)
{
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
    b->graph_n_work = -1;
}

// Interleave per-lattice item lists: lattice by lattice (order 0), or the
// largest lattices first with items interleaved across lattices (order 1).
template <typename I>
std::vector<I> order_items(std::vector<std::vector<I>>& per, int order)
{
    std::vector<I> w;
    if (order == 1) {
        std::vector<size_t> idx(per.size());
        for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
        std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return per[a].size() > per[b].size(); });
        size_t longest = idx.empty() ? 0 : per[idx[0]].size();
        for (size_t j = 0; j < longest; ++j)
            for (size_t i : idx)
                if (j < per[i].size()) w.push_back(per[i][j]);
    } else {
        for (auto& v : per) w.insert(w.end(), v.begin(), v.end());
    }
    return w;
}

// Global-load kernel: (lattice, first tile) items of tiles_per_item tiles.
std::vector<int2> build_work(const std::vector<pflbm_t*>& hs, const pflbm_schedule_t& s)
{
    const int G = std::max(1, s.tiles_per_item);
    std::vector<std::vector<int2>> per(hs.size());
    for (size_t i = 0; i < hs.size(); ++i) {
        int ntx = tiles_x(hs[i]->nx), nty = tiles_y(hs[i]->ny);
        for (int by = 0; by < nty; by += G)
            for (int bx = 0; bx < ntx; ++bx) per[i].push_back(make_int2((int)i, by * ntx + bx));
    }
    return order_items(per, s.order);
}

// Staged kernel: (lattice, strip, first block, blocks | shape << 16) items,
// shape and blocks per item by size class.
std::vector<int4> build_work_staged(const std::vector<pflbm_t*>& hs, const pflbm_schedule_t& s)
{
    std::vector<std::vector<int4>> per(hs.size());
    for (size_t i = 0; i < hs.size(); ++i) {
        const long long nodes = (long long)hs[i]->nx * hs[i]->ny;
        int shape = 0, L = std::max(1, s.tiles_per_item);
        for (int k = 0; k < std::min(8, s.n_classes); ++k)
            if (nodes <= s.class_max_nodes[k]) {
                shape = s.class_shape[k] == 1 ? 1 : 0;
                L = std::max(1, s.class_tiles[k]);
                break;
            }
        const int TXs = shape ? 64 : 32, TYs = shape ? 4 : 8;
        const int nsx = (hs[i]->nx + TXs - 1) / TXs, nby = (hs[i]->ny + TYs - 1) / TYs;
        L = std::min(L, std::min(nby, 0xffff));
        for (int b0 = 0; b0 < nby; b0 += L)
            for (int sx = 0; sx < nsx; ++sx)
                per[i].push_back(make_int4((int)i, sx, b0, std::min(L, nby - b0) | (shape << 16)));
    }
    return order_items(per, s.order);
}

int upload(pflbm_batch_t* b)
{
    const int n = (int)b->hs.size();
    std::vector<unsigned char> a0(b->args_bytes * n), a1(b->args_bytes * n);
    b->cur0.resize(n);
    b->nodes = 0;
    for (int i = 0; i < n; ++i) {
        pflbm_t* h = b->hs[i];
        write_step_args(h, 0, a0.data() + b->args_bytes * i);
        write_step_args(h, 1, a1.data() + b->args_bytes * i);
        b->cur0[i] = h->cur;
        b->nodes += (long long)h->nx * h->ny;
    }
    b->staged = b->precision != PFLBM_FP64 && b->sched.kernel == 2;
    for (pflbm_t* h : b->hs)
        if (!h->tma) b->staged = false;
    // the default kernel is the two-node one, one launch per group of
    // same-size lattices (measured fastest on mixes of small lattices in
    // FP32 and 16-bit storage)
    b->by_class = b->precision != PFLBM_FP64 && (b->sched.kernel == 3 || b->sched.kernel == 0);
    b->classes.clear();
    if (b->by_class) {
        // groups of lattices with the same size and viscosity mode, largest
        // first, each cut into launches of at most step2_class_capacity()
        const int K = step2_class_capacity(b->precision);
        std::vector<int> idx(n);
        for (int i = 0; i < n; ++i) idx[i] = i;
        auto vv = [&](int i) { return (b->hs[i]->prm.nu_l > 0 && b->hs[i]->prm.nu_g > 0) ? 1 : 0; };
        std::stable_sort(idx.begin(), idx.end(), [&](int p, int q) {
            const long long np = (long long)b->hs[p]->nx * b->hs[p]->ny, nq = (long long)b->hs[q]->nx * b->hs[q]->ny;
            if (np != nq) return np > nq;
            if (b->hs[p]->nx != b->hs[q]->nx) return b->hs[p]->nx > b->hs[q]->nx;
            return vv(p) < vv(q);
        });
        for (int j = 0; j < n;) {
            const pflbm_t* h0 = b->hs[idx[j]];
            int e = j;
            while (e < n && e - j < K && b->hs[idx[e]]->nx == h0->nx && b->hs[idx[e]]->ny == h0->ny &&
                   vv(idx[e]) == vv(idx[j]))
                ++e;
            pflbm_batch::ClassLaunch cl;
            cl.vv = vv(idx[j]);
            cl.nx = h0->nx;
            cl.ny = h0->ny;
            cl.count = e - j;
            for (int set = 0; set < 2; ++set) {
                const std::vector<unsigned char>& src = set ? a1 : a0;
                cl.descs[set].resize(b->args_bytes * cl.count);
                for (int m = 0; m < cl.count; ++m)
                    std::memcpy(cl.descs[set].data() + b->args_bytes * m, src.data() + b->args_bytes * idx[j + m],
                                b->args_bytes);
            }
            b->classes.push_back(std::move(cl));
            j = e;
        }
    }
    std::vector<unsigned char> wbytes;
    size_t item = b->staged ? sizeof(int4) : sizeof(int2);
    if (b->by_class) {
        // no work list: each launch's grid is (tiles, lattices)
    } else if (b->staged) {
        std::vector<int4> w4 = build_work_staged(b->hs, b->sched);
        wbytes.resize(w4.size() * item);
        if (!w4.empty()) std::memcpy(wbytes.data(), w4.data(), wbytes.size());
    } else {
        std::vector<int2> w2 = build_work(b->hs, b->sched);
        wbytes.resize(w2.size() * item);
        if (!w2.empty()) std::memcpy(wbytes.data(), w2.data(), wbytes.size());
    }
    const int n_items = (int)(wbytes.size() / item);
    if (n > b->cap_lattices) {
        int cap = std::max(n, 2 * b->cap_lattices);
        for (int k = 0; k < 2; ++k) {
            bfree(b, b->d_args[k], b->args_bytes * b->cap_lattices);
            b->d_args[k] = nullptr;
        }
        for (int k = 0; k < 2; ++k)
            if (int rc = balloc(b, &b->d_args[k], b->args_bytes * cap)) return rc;
        b->cap_lattices = cap;
        drop_graph(b);
    }
    if (n_items > b->cap_work) {
        int cap = std::max(n_items, 2 * b->cap_work);
        bfree(b, b->d_work, sizeof(int4) * b->cap_work);
        b->d_work = nullptr;
        void* p;
        if (int rc = balloc(b, &p, sizeof(int4) * cap)) return rc;
        b->d_work = p;
        b->cap_work = cap;
        drop_graph(b);
    }
    cudaError_t e = cudaMemcpyAsync(b->d_args[0], a0.data(), a0.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_args[1], a1.data(), a1.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !wbytes.empty())
        e = cudaMemcpyAsync(b->d_work, wbytes.data(), wbytes.size(), cudaMemcpyHostToDevice, b->stream);
    // the host vectors go out of scope on return: finish the copies first
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return set_error(PFLBM_ECUDA, cudaGetErrorString(e));
    drop_graph(b);   // kernel, work list or grid may differ from the captured ones
    b->n_work = n_items;
    b->phase = 0;
    int per_sm = b->staged ? staged_batch_ctas_per_sm(b->precision) : batch_max_ctas_per_sm(b->precision);
    if (b->sched.ctas_per_sm > 0) per_sm = std::min(per_sm, b->sched.ctas_per_sm);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    b->grid = std::max(1, std::min(b->n_work, std::max(1, per_sm) * std::max(1, sms)));
    if (b->by_class) {
        // info: the CTAs (one 64 x 8 tile each) of all launches, and the launches
        long long ctas = 0;
        for (const auto& cl : b->classes) ctas += (long long)cl.count * ((cl.nx + 63) / 64) * ((cl.ny + 7) / 8);
        b->n_work = (int)std::min(ctas, (long long)INT_MAX);
        b->grid = (int)b->classes.size();
    }
    if (b->by_class && b->classes.size() > 1) {
        // the forked streams and events of the per-class launches (made here,
        // outside any stream capture)
        const int nf = std::min((int)b->classes.size(), (int)pflbm_batch::kForks);
        for (int k = 0; k < nf; ++k) {
            cudaError_t e2 = cudaSuccess;
            if (!b->fork_stream[k]) e2 = cudaStreamCreateWithFlags(&b->fork_stream[k], cudaStreamNonBlocking);
            if (e2 == cudaSuccess && !b->join_ev[k])
                e2 = cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming);
            if (e2 != cudaSuccess) return set_error(PFLBM_ECUDA, cudaGetErrorString(e2));
        }
        if (!b->fork_ev) {
            cudaError_t e2 = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
            if (e2 != cudaSuccess) return set_error(PFLBM_ECUDA, cudaGetErrorString(e2));
        }
    }
    return PFLBM_OK;
}

int check_members(pflbm_t* const* hs, int count, int precision, int device, cudaStream_t stream)
{
    for (int i = 0; i < count; ++i) {
        if (!hs[i]) return set_error(PFLBM_EINVAL, "batch: NULL handle");
        if (hs[i]->precision != precision || hs[i]->device != device || hs[i]->stream != stream)
            return set_error(PFLBM_EINVAL, "batch: all handles need the same precision, device and stream");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return set_error(PFLBM_EINVAL, "batch: a handle appears twice");
    }
    return PFLBM_OK;
}

// Steps per captured graph (even). One graph replay runs each size group's
// steps back to back: measured on 256 small lattices (BF16, MLUPS) 46.8k with
// a join after every step, 47.6k at 2 steps per graph, 48.3k at 8, 47.9k at 32
// (300 steps), and over 400 steps 48.55k at 8 against 48.7k at 16. 8 divides
// the 200-step ticks of the server.
#ifndef PFLBM_BATCH_GRAPH_STEPS
#define PFLBM_BATCH_GRAPH_STEPS 8
#endif

cudaError_t launch_set(pflbm_batch_t* b, int set);

// nsteps steps from descriptor set `set0` on. With one launch per size group,
// each group takes its steps back to back on its own forked stream, and the
// streams join once at the end: a group's lattices need only their own
// previous step, so small groups run ahead instead of waiting each step for
// the largest.
cudaError_t launch_steps(pflbm_batch_t* b, int set0, int nsteps)
{
    const int nc = (int)b->classes.size();
    if (!b->by_class || nc <= 1) {
        cudaError_t e = cudaSuccess;
        for (int s = 0; s < nsteps && e == cudaSuccess; ++s) e = launch_set(b, (set0 + s) & 1);
        return e;
    }
    const int nf = std::min(nc, (int)pflbm_batch::kForks);
    cudaError_t e = cudaEventRecord(b->fork_ev, b->stream);
    for (int k = 0; k < nf && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->fork_stream[k], b->fork_ev, 0);
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
        const auto& cl = b->classes[c];
        for (int s = 0; s < nsteps && e == cudaSuccess; ++s)
            e = launch_step2_class(b->precision, cl.vv, cl.descs[(set0 + s) & 1].data(), cl.count, cl.nx, cl.ny,
                                   b->fork_stream[c % nf]);
    }
    for (int k = 0; k < nf && e == cudaSuccess; ++k) e = cudaEventRecord(b->join_ev[k], b->fork_stream[k]);
    for (int k = 0; k < nf && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->stream, b->join_ev[k], 0);
    return e;
}

cudaError_t launch_set(pflbm_batch_t* b, int set)
{
    if (b->staged)
        return launch_step_staged_batch(b->precision, b->d_args[set], (const int4*)b->d_work, b->n_work, b->grid,
                                        b->stream);
    if (b->by_class) {
        const int nc = (int)b->classes.size();
        if (nc == 1)
            return launch_step2_class(b->precision, b->classes[0].vv, b->classes[0].descs[set].data(),
                                      b->classes[0].count, b->classes[0].nx, b->classes[0].ny, b->stream);
        const int nf = std::min(nc, (int)pflbm_batch::kForks);   // streams made by upload()
        cudaError_t e = cudaEventRecord(b->fork_ev, b->stream);
        for (int k = 0; k < nf && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->fork_stream[k], b->fork_ev, 0);
        // largest groups first, dealt round-robin over the forked streams
        for (int c = 0; c < nc && e == cudaSuccess; ++c) {
            const auto& cl = b->classes[c];
            e = launch_step2_class(b->precision, cl.vv, cl.descs[set].data(), cl.count, cl.nx, cl.ny,
                                   b->fork_stream[c % nf]);
        }
        for (int k = 0; k < nf && e == cudaSuccess; ++k) e = cudaEventRecord(b->join_ev[k], b->fork_stream[k]);
        for (int k = 0; k < nf && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->stream, b->join_ev[k], 0);
        return e;
    }
    return launch_step_batch(b->precision, b->d_args[set], (const int2*)b->d_work, b->n_work,
                             std::max(1, b->sched.tiles_per_item), b->grid, b->stream);
}

int ensure_graph(pflbm_batch_t* b)
{
    if (b->graph_exec && b->graph_n_work == b->n_work) return PFLBM_OK;
    drop_graph(b);
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return set_error(PFLBM_ECUDA, cudaGetErrorString(e));
    cudaError_t e1 = launch_steps(b, 0, PFLBM_BATCH_GRAPH_STEPS);
    e = cudaStreamEndCapture(b->stream, &b->graph);
    if (e1 != cudaSuccess || e != cudaSuccess) {
        drop_graph(b);
        return set_error(PFLBM_ECUDA, "batch: graph capture failed");
    }
    e = cudaGraphInstantiate(&b->graph_exec, b->graph, 0);
    if (e != cudaSuccess) {
        drop_graph(b);
        return set_error(PFLBM_ECUDA, cudaGetErrorString(e));
    }
    b->graph_n_work = b->n_work;
    return PFLBM_OK;
}

}  // namespace

extern "C" {

void pflbm_schedule_default(pflbm_schedule_t* s)
{
    if (!s) return;
    std::memset(s, 0, sizeof(*s));
    s->ctas_per_sm = 0;
    s->tiles_per_item = 1;
    s->order = 0;
    s->use_graph = 1;
    s->kernel = 0;
    s->n_classes = 0;
}

int pflbm_batch_create(pflbm_batch_t** out, pflbm_t* const* hs, int count, const pflbm_schedule_t* sched)
{
    if (!out) return set_error(PFLBM_EINVAL, "batch: NULL out");
    *out = nullptr;
    if (!hs || count < 1) return set_error(PFLBM_EINVAL, "batch: need at least one handle");
    if (!hs[0]) return set_error(PFLBM_EINVAL, "batch: NULL handle");
    if (int rc = check_members(hs, count, hs[0]->precision, hs[0]->device, hs[0]->stream)) return rc;
    pflbm_batch_t* b = new pflbm_batch();
    b->precision = hs[0]->precision;
    b->device = hs[0]->device;
    b->stream = hs[0]->stream;
    // the batch's own small buffers come from cudaMalloc: a member's
    // allocator may belong to a handle that is destroyed while the batch lives
    pflbm_schedule_default(&b->sched);
    if (sched) b->sched = *sched;
    if (b->sched.tiles_per_item < 1) b->sched.tiles_per_item = 1;
    b->args_bytes = step_args_bytes(b->precision);
    b->hs.assign(hs, hs + count);
    DeviceGuard g(b->device);
    if (int rc = upload(b)) {
        pflbm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return PFLBM_OK;
}

int pflbm_batch_set(pflbm_batch_t* b, pflbm_t* const* hs, int count)
{
    if (!b || !hs || count < 1) return set_error(PFLBM_EINVAL, "batch: invalid arguments");
    if (int rc = check_members(hs, count, b->precision, b->device, b->stream)) return rc;
    DeviceGuard g(b->device);
    b->hs.assign(hs, hs + count);
    return upload(b);
}

int pflbm_batch_step(pflbm_batch_t* b, int64_t n)
{
    if (!b) return set_error(PFLBM_EINVAL, "batch: NULL batch");
    if (n < 0) return set_error(PFLBM_EINVAL, "batch: negative step count");
    if (n == 0) return PFLBM_OK;
    DeviceGuard g(b->device);
    NvtxRange range("pflbm_batch_step");
    bool stale = false;
    for (size_t i = 0; i < b->hs.size(); ++i) {
        pflbm_t* h = b->hs[i];
        if (h->hstatus && (h->hstatus[0] & 4))
            return set_error(PFLBM_ETIMEOUT, "batch: a wait for staged data in the step kernel gave up");
        if (h->hstatus && h->hstatus[0] != 0)
            return set_error(PFLBM_ENUMERIC, "batch: NaN or |u| >= 0.3 detected on the device");
        if (h->init_pending) {
            if (int rc = materialize_handle(h)) return rc;
        }
        if (h->cur != (b->cur0[i] ^ b->phase)) stale = true;
    }
    if (stale) {  // a member was stepped on its own: rewrite the descriptors
        if (int rc = upload(b)) return rc;
    }
    int64_t left = n;
    if (b->phase == 1) {
        cudaError_t e = launch_set(b, 1);
        if (e != cudaSuccess) return set_error(PFLBM_ECUDA, cudaGetErrorString(e));
        b->phase = 0;
        --left;
    }
    static_assert(PFLBM_BATCH_GRAPH_STEPS >= 2 && PFLBM_BATCH_GRAPH_STEPS % 2 == 0, "an even step count per graph");
    if (b->sched.use_graph && left >= PFLBM_BATCH_GRAPH_STEPS) {
        if (int rc = ensure_graph(b)) return rc;
        for (; left >= PFLBM_BATCH_GRAPH_STEPS; left -= PFLBM_BATCH_GRAPH_STEPS) {
            cudaError_t e = cudaGraphLaunch(b->graph_exec, b->stream);
            if (e != cudaSuccess) return set_error(PFLBM_ECUDA, cudaGetErrorString(e));
        }
    }
    while (left > 0) {
        cudaError_t e = launch_set(b, b->phase);
        if (e != cudaSuccess) return set_error(PFLBM_ECUDA, cudaGetErrorString(e));
        b->phase ^= 1;
        --left;
    }
    for (pflbm_t* h : b->hs) {
        if (n & 1) h->cur ^= 1;
        h->steps += n;
        h->replace_phi = true;
        if (int rc = post_status(h)) return rc;
    }
    // invariant: every member's current copy is cur0[i] ^ phase
    return PFLBM_OK;
}

int pflbm_batch_kernel(const pflbm_batch_t* b)
{
    if (!b) return set_error(PFLBM_EINVAL, "batch: NULL batch");
    return b->staged ? 2 : (b->by_class ? 3 : 1);
}

int pflbm_batch_info(const pflbm_batch_t* b, int* n_work, int* grid, int64_t* nodes)
{
    if (!b) return set_error(PFLBM_EINVAL, "batch: NULL batch");
    if (n_work) *n_work = b->n_work;
    if (grid) *grid = b->grid;
    if (nodes) *nodes = b->nodes;
    return PFLBM_OK;
}

void pflbm_batch_destroy(pflbm_batch_t* b)
{
    if (!b) return;
    DeviceGuard g(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (int k = 0; k < pflbm_batch::kForks; ++k) {
        if (b->fork_stream[k]) {
            cudaStreamSynchronize(b->fork_stream[k]);
            cudaStreamDestroy(b->fork_stream[k]);
        }
        if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    for (int k = 0; k < 2; ++k) bfree(b, b->d_args[k], b->args_bytes * b->cap_lattices);
    bfree(b, b->d_work, sizeof(int4) * b->cap_work);
    delete b;
}

}  // extern "C"
