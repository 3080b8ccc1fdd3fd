// Serving loop and autotuner.
//
// A scheduler thread owns the device work.  Submitted requests wait in a
// FIFO queue.  Whenever a launch slot is free it takes the longest prefix of
// the queue that fits the slot (at most max_requests_per_launch requests and
// the slot's ordering-flag arena), the in-flight limit and the memory budget,
// writes one launch descriptor (one segment per request) into the slot's
// pinned buffer and replays the slot's captured graph: descriptor copy,
// zero-fill, persistent fused kernel.  The kernel raises a flag in mapped host
// memory when a request's last work item is done; the scheduler turns flags
// into completions (timestamps, budget release).  Slots live on separate
// streams, so the next launch is already running while the previous one
// drains: requests that arrive while others run are admitted as soon as a
// slot and memory free up.
//
// Operators the multi-request kernel does not cover (3D FP32 or BF16x3, 2D
// with fft_size 64 or FP64, per-patch shapes) run their requests through the
// operator's own apply: a request at the head of the queue takes a free slot
// and, with the requests on the same operator and direction queued right
// behind it (up to kSoloMaxRhs right-hand sides), one apply on that slot's
// stream.  Several requests share the apply through a staging buffer of the
// slot: their x blocks are copied side by side, each starting at an even
// column so that its right-hand sides form the same pairs as alone (an odd
// block's last pair gets a zero column), and their y blocks are copied back,
// so each result is bitwise the request applied alone.  The apply's time is
// bounded below by the chain of ordering waits through the colours, so a
// batch of several small requests costs little more than one.  Such an
// operator has at most one launch in flight (its ordering flags and scratch
// volumes are per operator); different operators run concurrently on
// different slots.  The buffers such an apply grows on demand are grown by
// the scheduler thread just before the launch (the only thread that touches
// a served operator), which may synchronise the device once.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int64_t kFlagArenaWords = int64_t(1) << 22;   // ordering flags per launch slot
constexpr int kMaxInflightCap = 1024;
constexpr int32_t kSoloMaxRhs = 64;   // right-hand sides (staging columns) of one shared solo apply

struct Request {
    uint64_t ticket = 0;
    pc_operator *op = nullptr;
    int32_t nrhs = 0;
    const void *x = nullptr;
    void *y = nullptr;
    int64_t flag_words = 0;
    int64_t scratch_bytes = 0;
    double submit_s = 0, launch_s = 0, finish_s = 0;
    int state = 0;      // 0 queued, 1 launched, 2 done, 3 failed
    int status = PC_OK;
    int hslot = -1;     // host completion flag index
    int launch_requests = 0;
    bool solo = false;  // runs through the operator's own apply (not a batched 2D operator)
    bool adjoint = false;   // Y = A~* X (Eq. adjoint_random_z)
    // a launch slot still lists the request (until its launch ends); a
    // request polled before that is deleted by the slot, not by the poll
    bool attached = false;
    bool collected = false;
    std::string error;
};

struct LaunchSlot {
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr, graph_adj = nullptr;     // forward and adjoint launches
    cudaGraphExec_t exec = nullptr, exec_adj = nullptr;
    pc::LaunchDesc *h_desc = nullptr;   // pinned
    pc::LaunchDesc *d_desc = nullptr;
    uint32_t *d_flags = nullptr;
    uint32_t *d_seg_done = nullptr;
    unsigned long long *d_counter = nullptr;
    int32_t *d_status = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    bool solo = false;                  // running requests through their operator's own apply
    void *d_stage = nullptr;            // solo applies shared by several requests: x, then y columns
    int64_t stage_bytes = 0;
    std::vector<Request *> reqs;
};

}  // namespace

struct pc_server {
    pc_context *ctx = nullptr;
    pc_serve_config cfg{};
    std::mutex mu;
    std::condition_variable cv;
    std::thread th;
    bool stop = false;
    std::string fatal;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> all;
    uint64_t next_ticket = 1;
    std::vector<LaunchSlot> slots;
    uint32_t *h_flags = nullptr;        // mapped pinned host memory
    uint32_t *d_hflags = nullptr;
    std::vector<int> free_hslots;
    int64_t budget_used = 0, budget_peak = 0;
    std::unordered_map<pc_operator *, int> op_inflight;
    std::unordered_map<pc_operator *, int64_t> op_bytes;   // operator bytes counted while it has work in flight
    int inflight = 0;
    std::vector<double> latencies;
    int64_t rhs_done = 0, launches = 0;
    double first_submit = -1.0, last_finish = 0.0;
    Clock::time_point t0;
    int ctas = 0;
    size_t smem = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

pc_status srv_fail(pc_server *s, pc_status st, const std::string &msg) {
    if (s && s->ctx) s->ctx->last_error = msg;
    return st;
}

void release_budget(pc_server *s, Request *r) {
    s->budget_used -= r->scratch_bytes;
    auto it = s->op_inflight.find(r->op);
    if (it != s->op_inflight.end() && --it->second == 0) {
        s->budget_used -= s->op_bytes[r->op];
        s->op_bytes.erase(r->op);
        s->op_inflight.erase(it);
    }
    --s->inflight;
    if (r->hslot >= 0) s->free_hslots.push_back(r->hslot);
    r->hslot = -1;
}

// Bytes the request adds to the budget if admitted now.
int64_t admission_bytes(pc_server *s, const Request *r) {
    return r->scratch_bytes + (s->op_inflight.count(r->op) ? 0 : int64_t(r->op->device_bytes));
}

void reap(pc_server *s) {
    for (auto &sl : s->slots) {
        if (!sl.busy) continue;
        const double t = s->now();
        for (Request *r : sl.reqs) {
            // early completion through the mapped flag (batched 2D requests
            // only: a solo request has no flag slot and completes with its launch)
            if (r->state != 1 || r->hslot < 0) continue;
            if (reinterpret_cast<volatile uint32_t *>(s->h_flags)[r->hslot] != 0u) {
                r->state = 2;
                r->finish_s = t;
                s->latencies.push_back(r->finish_s - r->submit_s);
                s->rhs_done += r->nrhs;
                s->last_finish = t;
                release_budget(s, r);
            }
        }
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        // the launch has ended: anything not flagged failed.  A solo request
        // reports through its operator's timeout flag.
        int32_t status = 0;
        int32_t *d_status = sl.solo ? sl.reqs.front()->op->d_ctrl + 2 : sl.d_status;
        if (q == cudaSuccess &&
            cudaMemcpyAsync(&status, d_status, sizeof(status), cudaMemcpyDeviceToHost, sl.stream) == cudaSuccess)
            cudaStreamSynchronize(sl.stream);
        for (Request *r : sl.reqs) {
            if (r->state != 1) continue;
            // a launch that ended with a clean status has finished every item of
            // every request in it; the mapped-memory flags only report earlier
            if (q == cudaSuccess && !status) {
                r->state = 2;
                r->finish_s = s->now();
                s->latencies.push_back(r->finish_s - r->submit_s);
                s->rhs_done += r->nrhs;
                s->last_finish = r->finish_s;
            } else {
                r->state = 3;
                if (q != cudaSuccess) {
                    r->status = PC_ERR_CUDA;
                    r->error = std::string("launch failed: ") + cudaGetErrorString(q);
                } else if (status) {
                    r->status = PC_ERR_TIMEOUT;
                    r->error = status == 1 ? "a bounded overlap-order wait gave up"
                                           : "a bounded spectrum-copy wait gave up";
                }
            }
            release_budget(s, r);
        }
        if (status) cudaMemsetAsync(d_status, 0, sizeof(int32_t), sl.stream);
        for (Request *r : sl.reqs) {
            r->attached = false;
            if (r->collected) delete r;   // polled while the launch still ran
        }
        sl.reqs.clear();
        sl.busy = false;
        sl.solo = false;
    }
}

// The solo request at the head of the queue, with the requests on the same
// operator and direction right behind it, on slot sl.  Returns false if it
// has to wait (FIFO: nothing behind it overtakes).
bool launch_solo(pc_server *s, LaunchSlot &sl) {
    Request *r = s->queue.front();
    pc_operator *op = r->op;
    if (s->op_inflight.count(op)) return false;                 // one launch per solo operator
    if (s->inflight >= s->cfg.max_inflight) return false;
    std::vector<Request *> take{r};
    auto cols_of = [](const Request *q) { return q->nrhs + (q->nrhs & 1); };
    int32_t cols = cols_of(r);
    for (size_t i = 1; i < s->queue.size(); ++i) {
        Request *q = s->queue[i];
        if (q->op != op || q->adjoint != r->adjoint) break;
        if (int(take.size()) >= s->cfg.max_requests_per_launch) break;
        if (s->inflight + int(take.size()) >= s->cfg.max_inflight) break;
        if (cols + cols_of(q) > kSoloMaxRhs) break;
        take.push_back(q);
        cols += cols_of(q);
    }
    const int64_t N = op->N, el = op->elem;
    int64_t stage = take.size() > 1 ? 2 * int64_t(cols) * N * el : 0;
    if (stage && s->budget_used + admission_bytes(s, r) + stage > s->cfg.hbm_budget_bytes) {
        take.resize(1);   // the head request alone fits better than a shared apply
        stage = 0;
    }
    if (stage > sl.stage_bytes) {
        // the slot is idle: nothing of its own uses the old staging buffer
        cudaFree(sl.d_stage);
        sl.d_stage = nullptr;
        sl.stage_bytes = 0;
        if (cudaMalloc(&sl.d_stage, size_t(stage)) == cudaSuccess) {
            sl.stage_bytes = stage;
        } else {
            cudaGetLastError();
            take.resize(1);
            stage = 0;
        }
    }
    if (take.size() == 1) cols = r->nrhs;
    // Grow the operator's ordering flags and scratch for this launch here,
    // on the scheduler thread, the only thread that touches a served
    // operator.  Growing synchronises the device first, so no launch still
    // uses the buffers it frees.
    const pc_status pst = pc::prepare_batch(op, cols);
    if (pst != PC_OK) {
        s->queue.pop_front();
        r->state = 3;
        r->status = int(pst);
        r->error = op->ctx->last_error;
        return true;
    }
    if (s->budget_used + admission_bytes(s, r) + stage > s->cfg.hbm_budget_bytes) return false;
    s->budget_used += admission_bytes(s, r) + stage;
    s->op_bytes[op] = int64_t(op->device_bytes);
    r->scratch_bytes = stage;   // released with the head request
    const double t = s->now();
    for (Request *q : take) {
        s->op_inflight[op]++;
        ++s->inflight;
        s->queue.pop_front();
        q->state = 1;
        q->launch_s = t;
        q->launch_requests = int(take.size());
    }
    s->budget_peak = std::max(s->budget_peak, s->budget_used);
    auto apply = [&](const void *x, void *y, int32_t nrhs) {
        return r->adjoint ? pc_apply_adjoint_batched(op, nrhs, x, N, y, N, sl.stream)
                          : pc_apply_batched(op, nrhs, x, N, y, N, sl.stream);
    };
    pc_status st = PC_OK;
    cudaError_t e = cudaSuccess;
    if (take.size() == 1) {
        st = apply(r->x, r->y, r->nrhs);
    } else {
        char *xs = static_cast<char *>(sl.d_stage), *ys = xs + int64_t(cols) * N * el;
        int64_t off = 0;
        for (Request *q : take) {
            const int64_t bytes = int64_t(q->nrhs) * N * el;
            if (e == cudaSuccess) e = cudaMemcpyAsync(xs + off, q->x, size_t(bytes), cudaMemcpyDeviceToDevice, sl.stream);
            if (e == cudaSuccess && (q->nrhs & 1))
                e = cudaMemsetAsync(xs + off + bytes, 0, size_t(N * el), sl.stream);   // the odd block's partner
            off += int64_t(cols_of(q)) * N * el;
        }
        if (e == cudaSuccess) st = apply(xs, ys, cols);
        off = 0;
        for (Request *q : take) {
            if (e == cudaSuccess && st == PC_OK)
                e = cudaMemcpyAsync(q->y, ys + off, size_t(int64_t(q->nrhs) * N * el), cudaMemcpyDeviceToDevice,
                                    sl.stream);
            off += int64_t(cols_of(q)) * N * el;
        }
    }
    if (st == PC_OK && e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
    if (st != PC_OK || e != cudaSuccess) {
        for (Request *q : take) {
            q->state = 3;
            q->status = st != PC_OK ? int(st) : int(PC_ERR_CUDA);
            q->error = st != PC_OK ? op->ctx->last_error : std::string(cudaGetErrorString(e));
            release_budget(s, q);
        }
        return true;
    }
    sl.reqs = take;
    for (Request *q : take) q->attached = true;
    sl.busy = true;
    sl.solo = true;
    ++s->launches;
    return true;
}

void try_launch(pc_server *s) {
    for (auto &sl : s->slots) {
        if (sl.busy || s->queue.empty()) continue;
        if (s->queue.front()->solo) {
            if (!launch_solo(s, sl)) return;
            continue;
        }
        std::vector<Request *> take;
        int64_t words = 0, extra = 0;
        std::unordered_map<pc_operator *, int> seen;
        const bool adj = s->queue.front()->adjoint;
        for (Request *r : s->queue) {
            if (r->solo) break;   // the solo request takes a slot of its own next
            if (r->adjoint != adj) break;   // one direction per launch (FIFO: no overtaking)
            if (int(take.size()) >= s->cfg.max_requests_per_launch) break;
            if (s->inflight + int(take.size()) >= s->cfg.max_inflight) break;
            if (s->free_hslots.size() <= take.size()) break;
            if (words + r->flag_words > kFlagArenaWords) break;
            int64_t add = r->scratch_bytes;
            if (!s->op_inflight.count(r->op) && !seen.count(r->op)) add += int64_t(r->op->device_bytes);
            if (s->budget_used + extra + add > s->cfg.hbm_budget_bytes) break;   // FIFO: no overtaking
            take.push_back(r);
            seen[r->op] = 1;
            words += r->flag_words;
            extra += add;
        }
        if (take.empty()) return;
        pc::LaunchDesc &d = *sl.h_desc;
        std::memset(&d, 0, sizeof(pc::LaunchDesc));
        int64_t items = 0, woff = 0;
        const double t = s->now();
        for (size_t q = 0; q < take.size(); ++q) {
            Request *r = take[q];
            pc_operator *op = r->op;
            pc::Segment &sg = d.seg[q];
            const int32_t npairs = (r->nrhs + 1) / 2;
            pc::ApplyParams &p = sg.p;
            p.x = r->x;
            p.y = r->y;
            p.ldx = op->N;
            p.ldy = op->N;
            p.nrhs = r->nrhs;
            p.npairs = npairs;
            p.n[0] = int32_t(op->shape[0]);
            p.n[1] = int32_t(op->shape[1]);
            p.n[2] = int32_t(op->shape[2]);
            p.nx[0] = p.n[0];
            p.nx[1] = p.n[1];
            p.nx[2] = p.n[2];
            p.R = op->R;
            p.tiles = op->d_tiles;
            p.color_start = op->d_color_start;
            p.n_colors = op->n_colors;
            p.dep_start = op->d_dep_start;
            p.dep = op->d_dep;
            p.done = sl.d_flags + woff;
            p.done_ld = npairs;
            p.epoch = 1u;
            p.ctrl = nullptr;
            p.spec = op->d_spec;
            p.spec_stride = op->spec_stride;
            p.w = op->d_w;
            p.tw = op->d_tw;
            p.wait_ns = op->wait_ns;
            p.total_items = int64_t(op->n_tiles) * npairs;
            sg.item_begin = items;
            r->hslot = s->free_hslots.back();
            s->free_hslots.pop_back();
            reinterpret_cast<volatile uint32_t *>(s->h_flags)[r->hslot] = 0u;
            sg.slot = r->hslot;
            items += p.total_items;
            woff += r->flag_words;
            // admit
            if (!s->op_inflight.count(op)) {
                s->budget_used += int64_t(op->device_bytes);
                s->op_bytes[op] = int64_t(op->device_bytes);
            }
            s->op_inflight[op]++;
            s->budget_used += r->scratch_bytes;
            ++s->inflight;
            r->state = 1;
            r->launch_s = t;
            r->launch_requests = int(take.size());
        }
        std::atomic_thread_fence(std::memory_order_seq_cst);   // flag resets land before the launch
        d.nseg = int32_t(take.size());
        d.total_items = items;
        s->budget_peak = std::max(s->budget_peak, s->budget_used);
        for (size_t q = 0; q < take.size(); ++q) s->queue.pop_front();
        cudaError_t e = cudaGraphLaunch(adj ? sl.exec_adj : sl.exec, sl.stream);
        if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
        if (e != cudaSuccess) {
            s->fatal = std::string("graph launch: ") + cudaGetErrorString(e);
            for (Request *r : take) {
                r->state = 3;
                r->status = PC_ERR_CUDA;
                r->error = s->fatal;
                release_budget(s, r);
            }
            continue;
        }
        sl.reqs = take;
        for (Request *r : take) r->attached = true;
        sl.busy = true;
        ++s->launches;
    }
}

void scheduler(pc_server *s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        reap(s);
        if (!s->stop) try_launch(s);
        bool busy = false;
        for (auto &sl : s->slots) busy = busy || sl.busy;
        if (s->stop && !busy) break;
        if (!busy && s->queue.empty()) {
            s->cv.wait_for(lk, std::chrono::milliseconds(50));
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(10));
            lk.lock();
        }
    }
}

void free_server(pc_server *s) {
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
        if (sl.graph) cudaGraphDestroy(sl.graph);
        if (sl.exec_adj) cudaGraphExecDestroy(sl.exec_adj);
        if (sl.graph_adj) cudaGraphDestroy(sl.graph_adj);
        if (sl.h_desc) cudaFreeHost(sl.h_desc);
        cudaFree(sl.d_desc);
        cudaFree(sl.d_flags);
        cudaFree(sl.d_seg_done);
        cudaFree(sl.d_counter);
        cudaFree(sl.d_status);
        cudaFree(sl.d_stage);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->h_flags) cudaFreeHost(s->h_flags);
    for (auto &kv : s->all) delete kv.second;
    delete s;
}

}  // namespace

extern "C" {

pc_status pc_serve_create(pc_context *ctx, const pc_serve_config *cfg, pc_server **out) {
    if (!ctx || !cfg || !out) return PC_ERR_ARG;
    *out = nullptr;
    if (cfg->hbm_budget_bytes <= 0 || cfg->max_inflight < 1 || cfg->max_inflight > kMaxInflightCap ||
        cfg->streams < 1 || cfg->streams > 4 || cfg->max_requests_per_launch < 1 ||
        cfg->max_requests_per_launch > pc::kMaxSegments) {
        ctx->last_error = "invalid serving configuration";
        return PC_ERR_ARG;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        ctx->last_error = "cannot select the context's device";
        return PC_ERR_CUDA;
    }
    auto *s = new pc_server;
    s->ctx = ctx;
    s->cfg = *cfg;
    s->t0 = Clock::now();
    int per_sm = 0;
    cudaError_t e = pc::fft2d_configure(128, PC_FP32, &per_sm, &s->smem);
    s->ctas = ctx->num_sms * std::max(per_sm, 1);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&s->h_flags), sizeof(uint32_t) * kMaxInflightCap,
                                            cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->d_hflags), s->h_flags, 0);
    if (e == cudaSuccess) std::memset(s->h_flags, 0, sizeof(uint32_t) * kMaxInflightCap);
    for (int q = kMaxInflightCap - 1; q >= 0; --q) s->free_hslots.push_back(q);
    s->slots.resize(cfg->streams);
    for (auto &sl : s->slots) {
        if (e != cudaSuccess) break;
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&sl.h_desc), sizeof(pc::LaunchDesc), 0);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_desc, sizeof(pc::LaunchDesc));
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_flags, sizeof(uint32_t) * kFlagArenaWords);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_seg_done, sizeof(uint32_t) * pc::kMaxSegments);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_counter, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_status, sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMemsetAsync(sl.d_status, 0, sizeof(int32_t), sl.stream);
        if (e == cudaSuccess) std::memset(sl.h_desc, 0, sizeof(pc::LaunchDesc));
        // capture, forward and adjoint: descriptor upload, zero-fill, persistent fused kernel
        for (int adj = 0; adj < 2 && e == cudaSuccess; ++adj) {
            cudaGraph_t &g = adj ? sl.graph_adj : sl.graph;
            cudaGraphExec_t &x = adj ? sl.exec_adj : sl.exec;
            e = cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e1 = cudaMemcpyAsync(sl.d_desc, sl.h_desc, sizeof(pc::LaunchDesc), cudaMemcpyHostToDevice,
                                                 sl.stream);
                cudaError_t e2 = e1 == cudaSuccess
                                     ? pc::launch_round(sl.d_desc, sl.d_counter, sl.d_status, sl.d_seg_done,
                                                        s->d_hflags, s->ctas, s->smem, sl.stream, 128, PC_FP32,
                                                        adj == 1)
                                     : e1;
                e = cudaStreamEndCapture(sl.stream, &g);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
        }
    }
    if (e != cudaSuccess) {
        ctx->last_error = std::string("pc_serve_create: ") + cudaGetErrorString(e);
        free_server(s);
        return e == cudaErrorMemoryAllocation ? PC_ERR_NOMEM : PC_ERR_CUDA;
    }
    s->th = std::thread(scheduler, s);
    *out = s;
    return PC_OK;
}

pc_status pc_serve_submit(pc_server *s, pc_operator *op, int32_t nrhs, const void *x, void *y, uint32_t flags,
                          uint64_t *ticket) {
    if (!s || !ticket) return PC_ERR_ARG;
    if (!op || nrhs < 1 || !x || !y || (flags & ~PC_SERVE_ADJOINT) != 0)
        return srv_fail(s, PC_ERR_ARG, "bad request arguments");
    const bool adjoint = (flags & PC_SERVE_ADJOINT) != 0;
    if (op->ctx->device != s->ctx->device) return srv_fail(s, PC_ERR_ARG, "operator lives on another device");
    // the multi-request kernel covers 2D FP32 operators with fft_size 128;
    // every other operator runs its requests alone through its own apply
    const bool solo = op->d != 2 || op->prec != PC_FP32 || op->P != 128 || !op->parts.empty();
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) % op->elem)
        return srv_fail(s, PC_ERR_ARG, "x and y must be aligned to the element size");
    auto *r = new Request;
    r->op = op;
    r->nrhs = nrhs;
    r->x = x;
    r->y = y;
    r->solo = solo;
    r->adjoint = adjoint;
    // 2D: the request's ordering flags live in the launch slot's arena; 3D:
    // in the operator, whose scratch has already been counted in its size
    r->flag_words = solo ? 0 : int64_t(op->n_tiles) * ((nrhs + 1) / 2);
    r->scratch_bytes = solo ? 0 : r->flag_words * 4;
    if (r->flag_words > kFlagArenaWords) {
        delete r;
        return srv_fail(s, PC_ERR_BUDGET, "request needs more ordering flags than a launch slot holds; split it");
    }
    if (int64_t(op->device_bytes) + r->scratch_bytes > s->cfg.hbm_budget_bytes) {
        delete r;
        return srv_fail(s, PC_ERR_BUDGET, "operator and request exceed the serving budget");
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return srv_fail(s, PC_ERR_ARG, "server is stopping");
        }
        r->ticket = s->next_ticket++;
        r->submit_s = s->now();
        if (s->first_submit < 0) s->first_submit = r->submit_s;
        s->queue.push_back(r);
        s->all[r->ticket] = r;
        *ticket = r->ticket;
    }
    s->cv.notify_one();
    return PC_OK;
}

pc_status pc_serve_poll(pc_server *s, uint64_t ticket, pc_request_info *info) {
    if (!s) return PC_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->fatal.empty()) s->ctx->last_error = s->fatal;
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return srv_fail(s, PC_ERR_ARG, "unknown ticket");
    Request *r = it->second;
    if (r->state < 2) return PC_ERR_NOT_READY;
    if (info) {
        info->submit_s = r->submit_s;
        info->launch_s = r->launch_s;
        info->finish_s = r->finish_s;
        info->nrhs = r->nrhs;
        info->launch_requests = r->launch_requests;
        info->status = r->state == 2 ? PC_OK : r->status;
    }
    const pc_status st = r->state == 2 ? PC_OK : pc_status(r->status);
    const std::string msg = r->error;
    s->all.erase(it);
    // a request that completed early (its flag in mapped memory) is still on
    // its slot's list until the launch ends: the slot deletes it then
    if (r->attached)
        r->collected = true;
    else
        delete r;
    if (st != PC_OK) return srv_fail(s, st, msg);
    return PC_OK;
}

pc_status pc_serve_stats_get(pc_server *s, pc_serve_stats *st) {
    if (!s || !st) return PC_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(st, 0, sizeof(*st));
    st->completed = int64_t(s->latencies.size());
    st->rhs_completed = s->rhs_done;
    st->launches = s->launches;
    st->peak_bytes = s->budget_peak;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, size_t(q * double(v.size() - 1) + 0.5))]; };
        st->p50_latency_s = pct(0.50);
        st->p99_latency_s = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_latency_s = sum / double(v.size());
        st->busy_s = s->last_finish - s->first_submit;
        st->rhs_per_s = st->busy_s > 0 ? double(s->rhs_done) / st->busy_s : 0.0;
    }
    return PC_OK;
}

pc_status pc_serve_destroy(pc_server *s) {
    if (!s) return PC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_one();
    if (s->th.joinable()) s->th.join();
    free_server(s);
    return PC_OK;
}

}  // extern "C"
