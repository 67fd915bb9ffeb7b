// Serving runtime: continuous batching of BICGK / ATAX / GEMVER / GESUMMV
// requests (Table I) over resident operands, with the scheduling loop in
// native code so that a launch costs the host a few microseconds.
//
// The loop (one host thread, polling):
//   - requests whose arrival time has passed join a FIFO;
//   - completions: each launch slot (a caller stream) records an event after
//     its work and an asynchronous copy of the launch's device status word
//     into pinned memory; a finished slot stamps its requests' completion
//     time and status and returns their memory to the arena;
//   - admission, for every free slot: a request with n >= direct_n runs alone
//     through its single-instance reduced-precision entry point (its sweep
//     spreads one matrix over every SM); otherwise requests from the head of
//     the FIFO form a batch (up to max_batch, stopping before the next direct
//     one) whose outputs and workspace fit the arena, planned once and
//     submitted through the batched form;
//   - a request that cannot fit even with nothing in flight is rejected with
//     BTO_ERR_BUDGET.
// Memory: every output vector, GEMVER's B and every workspace comes from the
// caller's device arena (the HBM budget) through a first-fit allocator with
// coalescing; nothing is allocated on the device by the runtime.
#include "check.cuh"
#include "arena.h"
#include <algorithm>
#include <chrono>
#include <deque>
#include <iterator>
#include <map>
#include <thread>
#include <vector>

namespace bto {
namespace {

constexpr size_t kGranule = kArenaGranule;

struct Block {
    size_t off = 0, bytes = 0;
    bool on = false;
};

struct Slot {
    cudaEvent_t ev = nullptr;
    bool busy = false;
    std::vector<int64_t> reqs;
    Block ws;
};

int n_outputs(int op) { return (op == BTO_OP_BICGK || op == BTO_OP_GEMVER) ? 2 : 1; }
int n_inputs(int op) { return op == BTO_OP_BICGK ? 2 : op == BTO_OP_GEMVER ? 6 : 1; }
size_t esize(int a_type) { return a_type == BTO_BF16 ? 2 : 4; }
int tix(int a_type) { return a_type == BTO_BF16 ? 1 : 0; }

class Server {
 public:
    Server(const bto_serve_cfg& c, int64_t count, const bto_serve_req* rq, bto_serve_res* res)
        : c_(c), count_(count), rq_(rq), res_(res), arena_(c.arena_bytes), base_(static_cast<char*>(c.arena)),
          blocks_(count), slots_(c.nstreams) {}

    ~Server() {
        for (Slot& s : slots_)
            if (s.ev) cudaEventDestroy(s.ev);
        if (plan_) batch_plan_destroy(plan_);
    }

    bto_status run(bto_serve_stats* stats) {
        if (!device_info(&dev_)) return BTO_ERR_CUDA;
        for (Slot& s : slots_)
            if (cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess) return BTO_ERR_CUDA;
        plan_ = batch_plan_create();
        // Pinned staging: slot status words first, then one plan buffer per slot.
        if (c_.staging && c_.staging_bytes >= kGranule * 2) {
            status_ = static_cast<int*>(c_.staging);
            stage_each_ = (c_.staging_bytes - kGranule) / c_.nstreams / kGranule * kGranule;
        }
        for (int64_t i = 0; i < count_; i++) {
            res_[i].admit = res_[i].done = -1.0;
            res_[i].out[0] = res_[i].out[1] = res_[i].out[2] = -1;
            res_[i].status = BTO_OK;
            res_[i].direct = 0;
        }
        descs_.reserve(c_.max_batch);
        t0_ = std::chrono::steady_clock::now();
        int64_t next = 0;
        bool closed = false;
        double last = 0.0;
        for (;;) {
            const double tn = now();
            if (tn - last > dg_.max_gap_s) {
                dg_.max_gap_s = tn - last;
                dg_.max_gap_at_s = tn;
                gap_mark_ = true;
            }
            last = tn;
            if (c_.max_wall > 0 && tn > c_.max_wall) closed = true;
            while (!closed && next < count_ && rq_[next].t <= tn) pending_.push_back(next++);
            dg_.max_fifo = std::max<int64_t>(dg_.max_fifo, (int64_t)pending_.size());
            if (gap_mark_) {
                dg_.fifo_at_max_gap = (int64_t)pending_.size();
                gap_mark_ = false;
            }
            const double tc = now();
            const bool progressed = complete();
            dg_.max_complete_s = std::max(dg_.max_complete_s, now() - tc);
            bool launched = false;
            for (int si = 0; si < c_.nstreams && !pending_.empty(); si++)
                if (!slots_[si].busy) {
                    const double ta = now();
                    const bool ok = admit(si);
                    dg_.max_admit_s = std::max(dg_.max_admit_s, now() - ta);
                    if (!ok) break;
                    launched = true;
                }
            const bool idle = std::none_of(slots_.begin(), slots_.end(), [](const Slot& s) { return s.busy; });
            if (idle && pending_.empty() && (closed || next >= count_)) break;
            if (!progressed && !launched && idle && pending_.empty() && next < count_) {
                // Nothing to do before the next arrival.
                const double gap = rq_[next].t - now();
                if (gap > 300e-6) {
                    const double want = gap - 200e-6, ts = now();
                    std::this_thread::sleep_for(std::chrono::duration<double>(want));
                    dg_.max_oversleep_s = std::max(dg_.max_oversleep_s, now() - ts - want);
                    dg_.sleeps++;
                }
            }
        }
        stats->wall_s = now();
        stats->max_gap_s = dg_.max_gap_s;
        stats->max_gap_at_s = dg_.max_gap_at_s;
        stats->max_admit_s = dg_.max_admit_s;
        stats->max_complete_s = dg_.max_complete_s;
        stats->max_oversleep_s = dg_.max_oversleep_s;
        stats->max_fifo = dg_.max_fifo;
        stats->fifo_at_max_gap = dg_.fifo_at_max_gap;
        stats->sleeps = dg_.sleeps;
        stats->blocking_copies = dg_.blocking_copies;
        stats->max_query_s = dg_.max_query_s;
        stats->served = served_;
        stats->batches = batches_;
        stats->direct = direct_;
        stats->rejected = rejected_;
        stats->peak_bytes = (double)arena_.peak();
        return failed_;
    }

 private:
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0_).count();
    }

    bool direct(int64_t i) const { return c_.direct_n > 0 && rq_[i].n >= c_.direct_n; }

    bool take(size_t bytes, Block* b) {
        b->bytes = bytes;
        b->on = arena_.alloc(bytes, &b->off);
        return b->on;
    }
    void give(Block* b) {
        if (b->on) arena_.release(b->off, b->bytes);
        b->on = false;
    }

    // Leading dimension of GEMVER's B: n rounded up to 8 elements, so that its
    // columns start on 16-byte boundaries and both passes run TMA-fed (with
    // ld n, most n sent them to the load-instruction kernel, 3 to 10 times
    // slower at n >= 1500).
    static int64_t b_ld(int64_t n) { return (n + 7) / 8 * 8; }

    // Output vectors (and GEMVER's B) of request i.
    bool take_outputs(int64_t i) {
        const bto_serve_req& r = rq_[i];
        Blocks& bl = blocks_[i];
        for (int k = 0; k < n_outputs(r.op); k++)
            if (!take((size_t)r.n * sizeof(float), &bl.out[k])) { give_outputs(i); return false; }
        if (r.op == BTO_OP_GEMVER && !take((size_t)r.n * b_ld(r.n) * esize(r.a_type), &bl.out[2])) {
            give_outputs(i);
            return false;
        }
        return true;
    }
    void give_outputs(int64_t i) {
        for (Block& b : blocks_[i].out) give(&b);
    }
    void* at(const Block& b) const { return base_ + b.off; }

    // Either the front request is rejected (nothing in flight could make room) or admission waits.
    bool cannot_fit() {
        if (std::any_of(slots_.begin(), slots_.end(), [](const Slot& s) { return s.busy; })) return false;
        const int64_t i = pending_.front();
        pending_.pop_front();
        res_[i].status = BTO_ERR_BUDGET;
        res_[i].admit = res_[i].done = now();
        rejected_++;
        return true;
    }

    void stamp_admit(int64_t i, int path) {
        res_[i].admit = now();
        res_[i].direct = path;
        for (int k = 0; k < 3; k++) res_[i].out[k] = blocks_[i].out[k].on ? (int64_t)blocks_[i].out[k].off : -1;
    }

    // Enqueues the status copy and the completion event of slot si.
    void arm(int si, cudaStream_t st) {
        Slot& s = slots_[si];
        if (status_) {
            status_[si] = BTO_OK;
            cudaMemcpyAsync(&status_[si], at(s.ws), sizeof(int), cudaMemcpyDeviceToHost, st);
        }
        cudaEventRecord(s.ev, st);
        s.busy = true;
    }

    // A launch that failed on the host: its requests end now with that status.
    void fail_now(int si, bto_status e) {
        Slot& s = slots_[si];
        const double td = now();
        for (int64_t i : s.reqs) {
            res_[i].done = td;
            res_[i].status = e;
            give_outputs(i);
        }
        give(&s.ws);
        s.reqs.clear();
        if (failed_ == BTO_OK) failed_ = e;
    }

    bool admit(int si) {
        Slot& s = slots_[si];
        cudaStream_t st = (cudaStream_t)c_.streams[si];
        const int64_t i = pending_.front();
        if (direct(i)) {
            const bto_serve_req& r = rq_[i];
            WsLayout L;
            if (ws_layout(r.op, BTO_FORM_FUSED, r.n, r.n, r.a_type, dev_, &L) != BTO_OK) {
                pending_.pop_front();
                res_[i].status = BTO_ERR_UNSUPPORTED;
                res_[i].admit = res_[i].done = now();
                return true;
            }
            if (!take_outputs(i)) return cannot_fit();
            if (!take(std::max<size_t>(L.total, kGranule), &s.ws)) { give_outputs(i); return cannot_fit(); }
            pending_.pop_front();
            s.reqs.assign(1, i);
            stamp_admit(i, 1);
            const bto_status e = launch_direct(i, st, at(s.ws), s.ws.bytes);
            if (e != BTO_OK) { fail_now(si, e); return true; }
            arm(si, st);
            direct_++;
            return true;
        }
        descs_.clear();
        s.reqs.clear();
        while (!pending_.empty() && (int)s.reqs.size() < c_.max_batch) {
            const int64_t j = pending_.front();
            if (direct(j) || !take_outputs(j)) break;
            pending_.pop_front();
            s.reqs.push_back(j);
            descs_.push_back(desc(j));
        }
        if (s.reqs.empty()) return cannot_fit();
        size_t wsb = 0;
        for (;;) {
            if (!batch_plan_build(plan_, (int)s.reqs.size(), descs_.data(), c_.tile_cols, &wsb)) {
                fail_now(si, BTO_ERR_INVALID_VALUE);
                return true;
            }
            if (take(wsb, &s.ws)) break;
            // Give the last member back until the workspace fits.
            const int64_t j = s.reqs.back();
            s.reqs.pop_back();
            descs_.pop_back();
            give_outputs(j);
            pending_.push_front(j);
            if (s.reqs.empty()) return cannot_fit();
        }
        for (int64_t j : s.reqs) stamp_admit(j, 0);
        void* stage = status_ ? static_cast<char*>(c_.staging) + kGranule + (size_t)si * stage_each_ : nullptr;
        if (!stage || batch_plan_image_bytes(plan_) > stage_each_) dg_.blocking_copies++;
        const bto_status e = batch_plan_submit(plan_, at(s.ws), s.ws.bytes, stage, stage_each_, st);
        if (e != BTO_OK) { fail_now(si, e); return true; }
        arm(si, st);
        batches_++;
        return true;
    }

    bto_batch_desc desc(int64_t i) {
        const bto_serve_req& r = rq_[i];
        const Blocks& bl = blocks_[i];
        bto_batch_desc d{};
        d.op = r.op;
        d.a_type = r.a_type;
        d.m = d.n = r.n;
        d.lda = d.ldb = c_.nmax;
        d.alpha = c_.alpha;
        d.beta = c_.beta;
        d.A = c_.A[tix(r.a_type)][0];
        if (r.op == BTO_OP_GESUMMV) d.B = const_cast<void*>(c_.A[tix(r.a_type)][1]);
        if (r.op == BTO_OP_GEMVER) { d.B = at(bl.out[2]); d.ldb = b_ld(r.n); }
        for (int k = 0; k < n_inputs(r.op); k++) d.in[k] = c_.vec[k];
        for (int k = 0; k < n_outputs(r.op); k++) d.out[k] = static_cast<float*>(at(bl.out[k]));
        return d;
    }

    bto_status launch_direct(int64_t i, cudaStream_t st, void* ws, size_t wsb) {
        const bto_serve_req& r = rq_[i];
        const Blocks& bl = blocks_[i];
        const int64_t n = r.n, ld = c_.nmax;
        const void* A = c_.A[tix(r.a_type)][0];
        const float* const* v = c_.vec;
        float* o0 = static_cast<float*>(at(bl.out[0]));
        bto_stream_t s = (bto_stream_t)st;
        switch (r.op) {
            case BTO_OP_BICGK:
                return bto_bicgk_ex(n, n, r.a_type, A, ld, v[0], v[1], o0, static_cast<float*>(at(bl.out[1])), ws, wsb, s);
            case BTO_OP_GEMVER:
                return bto_gemver_ex(n, n, c_.alpha, c_.beta, r.a_type, A, ld, v[0], v[1], v[2], v[3], v[4], v[5],
                                     at(bl.out[2]), b_ld(n), o0, static_cast<float*>(at(bl.out[1])), ws, wsb, s);
            case BTO_OP_ATAX:
                return bto_atax_ex(n, n, c_.beta, r.a_type, A, ld, v[0], o0, ws, wsb, s);
            default:
                return bto_gesummv_ex(n, n, c_.alpha, c_.beta, r.a_type, A, ld, c_.A[tix(r.a_type)][1], ld, v[0], o0,
                                      ws, wsb, s);
        }
    }

    // Finished slots: stamp, read the status, release memory.
    bool complete() {
        bool any = false;
        for (int si = 0; si < c_.nstreams; si++) {
            Slot& s = slots_[si];
            if (!s.busy) continue;
            const double tq = now();
            const cudaError_t q = cudaEventQuery(s.ev);
            dg_.max_query_s = std::max(dg_.max_query_s, now() - tq);
            if (q == cudaErrorNotReady) continue;
            const double td = now();
            int status = BTO_OK;
            if (q != cudaSuccess) {
                cudaGetLastError();
                status = BTO_ERR_CUDA;
            } else if (status_) {
                status = status_[si];
            } else if (cudaMemcpy(&status, at(s.ws), sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                status = BTO_ERR_CUDA;
            }
            for (int64_t i : s.reqs) {
                res_[i].done = td;
                res_[i].status = status;
                served_++;
                if (!c_.keep_results) give_outputs(i);
            }
            if (status != BTO_OK && failed_ == BTO_OK) failed_ = (bto_status)status;
            give(&s.ws);
            s.reqs.clear();
            s.busy = false;
            any = true;
        }
        return any;
    }

    struct Blocks {
        Block out[3];
    };

    const bto_serve_cfg& c_;
    const int64_t count_;
    const bto_serve_req* rq_;
    bto_serve_res* res_;
    Arena arena_;
    char* base_;
    std::vector<Blocks> blocks_;
    std::vector<Slot> slots_;
    std::deque<int64_t> pending_;
    std::vector<bto_batch_desc> descs_;
    BatchPlan* plan_ = nullptr;
    DeviceInfo dev_{};
    int* status_ = nullptr;
    size_t stage_each_ = 0;
    std::chrono::steady_clock::time_point t0_;
    int64_t served_ = 0, batches_ = 0, direct_ = 0, rejected_ = 0;
    bto_serve_stats dg_{};   // diagnostics only
    bool gap_mark_ = false;
    bto_status failed_ = BTO_OK;
};

bool valid_req(const bto_serve_req& r, const bto_serve_cfg& c) {
    if (r.op != BTO_OP_BICGK && r.op != BTO_OP_ATAX && r.op != BTO_OP_GEMVER && r.op != BTO_OP_GESUMMV) return false;
    if (r.a_type != BTO_F32 && r.a_type != BTO_BF16) return false;
    if (r.n < 1 || r.n > c.nmax || !(r.t >= 0.0)) return false;
    if (!c.A[tix(r.a_type)][0] || (r.op == BTO_OP_GESUMMV && !c.A[tix(r.a_type)][1])) return false;
    for (int k = 0; k < n_inputs(r.op); k++)
        if (!c.vec[k]) return false;
    return true;
}

}  // namespace
}  // namespace bto

using namespace bto;

extern "C" bto_status bto_serve_run(const bto_serve_cfg* cfg, int64_t count, const bto_serve_req* req,
                                    bto_serve_res* res, bto_serve_stats* stats) {
    clear_invalid_arg();
    if (!cfg) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    const bto_serve_cfg& c = *cfg;
    const bool cfg_ok = c.nstreams >= 1 && c.nstreams <= 64 && c.streams && c.arena &&
                        (reinterpret_cast<uintptr_t>(c.arena) % kGranule) == 0 && c.max_batch >= 1 &&
                        c.tile_cols >= 16 && c.tile_cols <= 1024 && c.tile_cols % 16 == 0 && c.nmax >= 1 &&
                        c.direct_n >= 0 && c.max_wall >= 0.0 &&
                        (!c.staging || (reinterpret_cast<uintptr_t>(c.staging) % kGranule) == 0);
    if (!cfg_ok) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (count < 0) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (count > 0 && !req) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    for (int64_t i = 0; i < count; i++)
        if (!valid_req(req[i], c) || (i > 0 && req[i].t < req[i - 1].t)) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    if (count > 0 && !res) { set_invalid_arg(4); return BTO_ERR_INVALID_VALUE; }
    if (!stats) { set_invalid_arg(5); return BTO_ERR_INVALID_VALUE; }
    *stats = bto_serve_stats{};
    Server s(c, count, req, res);
    return s.run(stats);
}
