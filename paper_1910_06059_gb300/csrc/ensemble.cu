// Batched ensembles: many independent models (permeability realisations of
// uneven size) advanced together on one GPU.  Each member keeps its own
// Newton loop, time-step control, factorisation and BiCGStab graphs (the
// method of arXiv 1910.06059 Section 2.3 per member); the ensemble runs the
// members concurrently from a pool of host workers, each with its own CUDA
// stream, so the small members' latency-bound kernels (wavefront sweeps of
// nx + ny + nz levels, short vector kernels) overlap on the SMs instead of
// running one member at a time.
//
// Schedule: members are handed out largest first (the longest jobs start
// first, so the pool finishes together), or in the caller's order; the
// number of concurrent streams and the order are picked by an autotuner that
// times a short probe step of the real ensemble for each candidate and puts
// the members' states back after each probe.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

using bo::set_last_error;

struct bo_ensemble {
    std::vector<bo_sim*> members;
    std::vector<cudaStream_t> streams;
    int active = 1;                  // streams in use
    bool largest_first = true;
    int device = 0;
    // device time of a step: every worker stream waits on ev_start before its
    // first member and records ev_done[w] after its last; tstream joins them
    cudaStream_t tstream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;
    std::vector<cudaEvent_t> ev_done;
    double last_ms = -1.0;
};

namespace {

struct Snapshot {
    std::vector<double> p, sw, x, bhp;
    std::vector<unsigned char> flag;
    double dt_next = 0.0;
};

bo_status snapshot(bo_sim* m, Snapshot& s) {
    const int n = m->geo.n;
    s.p.resize(n);
    s.sw.resize(n);
    s.x.resize(n);
    s.flag.resize(n);
    s.bhp.resize(std::max(m->nw, 1));
    bo_status st = bo_get_state(m, s.p.data(), s.sw.data(), s.x.data(), s.flag.data(), s.bhp.data());
    if (st != BO_OK) return st;
    return bo_get_step_control(m, &s.dt_next);
}

bo_status restore(bo_sim* m, const Snapshot& s) {
    bo_status st = bo_set_state(m, s.p.data(), s.sw.data(), s.x.data(), s.flag.data(), s.bhp.data());
    if (st != BO_OK) return st;
    return bo_set_step_control(m, s.dt_next);
}

// One report step of every member with e->active workers; per-member
// statuses and reports (either may be null).
void run_step(bo_ensemble* e, double dt, const bo_newton_opts* opts, bo_step_report* reports,
              bo_status* statuses) {
    const int count = (int)e->members.size();
    std::vector<int> order(count);
    for (int q = 0; q < count; ++q) order[q] = q;
    if (e->largest_first)
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return e->members[a]->geo.n > e->members[b]->geo.n;
        });
    std::atomic<int> next{0};
    int nworkers = std::max(1, std::min(e->active, count));
    // streams are created on first use (one per worker, kept for later steps)
    for (int w = 0; w < nworkers; ++w)
        if (e->streams[w] == nullptr &&
            cudaStreamCreateWithFlags(&e->streams[w], cudaStreamNonBlocking) != cudaSuccess) {
            e->streams[w] = nullptr;
            nworkers = std::max(1, w);   // run with the streams that exist
            break;
        }
    if (e->streams[0] == nullptr) {
        for (int q = 0; q < count; ++q)
            if (statuses) statuses[q] = BO_ERR_CUDA;
        return;
    }
    // device-side bracket of the whole step (events of this ensemble)
    bool timed = e->ev_start != nullptr ||
                 (cudaStreamCreateWithFlags(&e->tstream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreate(&e->ev_start) == cudaSuccess &&
                  cudaEventCreate(&e->ev_end) == cudaSuccess);
    if (timed && (int)e->ev_done.size() < nworkers) {
        for (int w = (int)e->ev_done.size(); w < nworkers; ++w) {
            cudaEvent_t ev = nullptr;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                timed = false;
                break;
            }
            e->ev_done.push_back(ev);
        }
    }
    timed = timed && cudaEventRecord(e->ev_start, e->tstream) == cudaSuccess;
    e->last_ms = -1.0;
    auto work = [&](int w) {
        cudaSetDevice(e->device);
        cudaStream_t st = e->streams[w];
        if (timed) cudaStreamWaitEvent(st, e->ev_start, 0);
        for (;;) {
            const int q = next.fetch_add(1);
            if (q >= count) break;
            const int id = order[q];
            bo_sim* m = e->members[id];
            cudaStream_t own = m->stream;
            m->stream = st;
            bo_step_report rep{};
            const bo_status s = bo_step(m, dt, opts, &rep);
            m->stream = own;
            if (reports) reports[id] = rep;
            if (statuses) statuses[id] = s;
        }
        if (timed) cudaEventRecord(e->ev_done[w], st);
    };
    std::vector<std::thread> pool;
    pool.reserve(nworkers);
    try {
        for (int w = 1; w < nworkers; ++w) pool.emplace_back(work, w);
    } catch (const std::exception&) {
        // fewer threads than asked for: the members are shared through the
        // counter, so the workers that did start (and this thread) do them all
    }
    work(0);
    for (auto& t : pool) t.join();
    if (timed) {
        for (int w = 0; w < nworkers; ++w) cudaStreamWaitEvent(e->tstream, e->ev_done[w], 0);
        float ms = 0.f;
        if (cudaEventRecord(e->ev_end, e->tstream) == cudaSuccess &&
            cudaEventSynchronize(e->ev_end) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e->ev_start, e->ev_end) == cudaSuccess)
            e->last_ms = ms;
    }
}

}  // namespace

extern "C" {

bo_status bo_ensemble_create(bo_sim* const* members, int count, int streams, bo_ensemble** out) {
    if (out == nullptr || members == nullptr || count < 1 || streams < 1 || streams > 256)
        return set_last_error(BO_ERR_INVALID_ARG,
                              "bo_ensemble_create: NULL argument, count < 1 or streams not in 1..256");
    for (int q = 0; q < count; ++q)
        if (members[q] == nullptr || !members[q]->props_set)
            return set_last_error(BO_ERR_STATE, "bo_ensemble_create: member " + std::to_string(q) +
                                                    " is NULL or has no properties");
    for (int q = 0; q < count; ++q)
        for (int r = q + 1; r < count; ++r)
            if (members[q] == members[r])
                return set_last_error(BO_ERR_INVALID_ARG, "bo_ensemble_create: member " +
                                                              std::to_string(r) + " repeats member " +
                                                              std::to_string(q));
    auto* e = new bo_ensemble();
    e->members.assign(members, members + count);
    if (cudaGetDevice(&e->device) != cudaSuccess) {
        delete e;
        return set_last_error(BO_ERR_CUDA, "bo_ensemble_create: cudaGetDevice failed");
    }
    e->streams.assign(256, nullptr);   // created on first use
    e->active = streams;
    *out = e;
    return BO_OK;
}

bo_status bo_ensemble_set_schedule(bo_ensemble* e, int streams, int largest_first) {
    if (e == nullptr || streams < 1 || streams > 256)
        return set_last_error(BO_ERR_INVALID_ARG,
                              "bo_ensemble_set_schedule: NULL ensemble or streams not in 1..256");
    e->active = streams;
    e->largest_first = largest_first != 0;
    return BO_OK;
}

bo_status bo_ensemble_get_schedule(const bo_ensemble* e, int* streams, int* largest_first) {
    if (e == nullptr) return set_last_error(BO_ERR_INVALID_ARG, "bo_ensemble_get_schedule: NULL ensemble");
    if (streams) *streams = e->active;
    if (largest_first) *largest_first = e->largest_first ? 1 : 0;
    return BO_OK;
}

bo_status bo_ensemble_step(bo_ensemble* e, double dt, const bo_newton_opts* opts,
                           bo_step_report* reports, bo_status* statuses) {
    if (e == nullptr || !(dt > 0.0))
        return set_last_error(BO_ERR_INVALID_ARG, "bo_ensemble_step: NULL ensemble or dt <= 0");
    const int count = (int)e->members.size();
    std::vector<bo_status> st(count, BO_OK);
    try {
        run_step(e, dt, opts, reports, st.data());
    } catch (const std::exception&) {   // no memory for the schedule's vectors
        return set_last_error(BO_ERR_STATE, "bo_ensemble_step: out of host memory");
    }
    bo_status first = BO_OK;
    int failed = 0;
    for (int q = 0; q < count; ++q) {
        if (statuses) statuses[q] = st[q];
        if (st[q] != BO_OK) {
            if (first == BO_OK) {
                first = st[q];
                set_last_error(first, "bo_ensemble_step: member " + std::to_string(q) +
                                          " failed with status " + std::to_string((int)first));
            }
            ++failed;
        }
    }
    if (failed > 1)
        set_last_error(first, "bo_ensemble_step: " + std::to_string(failed) +
                                  " members failed; the first with status " +
                                  std::to_string((int)first) + " (per-member statuses in statuses[])");
    return first;
}

bo_status bo_ensemble_autotune(bo_ensemble* e, double dt_probe, const bo_newton_opts* opts,
                               const int* candidates, int ncand, double* seconds) {
    if (e == nullptr || candidates == nullptr || ncand < 1 || !(dt_probe > 0.0))
        return set_last_error(BO_ERR_INVALID_ARG,
                              "bo_ensemble_autotune: NULL argument, ncand < 1 or dt_probe <= 0");
    for (int c = 0; c < ncand; ++c)
        if (candidates[c] < 1 || candidates[c] > 256)
            return set_last_error(BO_ERR_INVALID_ARG,
                                  "bo_ensemble_autotune: a candidate is not in 1..256 streams");
    const int count = (int)e->members.size();
    std::vector<Snapshot> snap(count);
    for (int q = 0; q < count; ++q) {
        bo_status s = snapshot(e->members[q], snap[q]);
        if (s != BO_OK) return s;
    }
    double best = 1e300;
    int best_w = e->active;
    bool best_lf = e->largest_first;
    for (int order = 0; order < 2; ++order) {
        for (int c = 0; c < ncand; ++c) {
            e->active = candidates[c];
            e->largest_first = order == 0;
            std::vector<bo_status> st(count, BO_OK);
            const auto t0 = std::chrono::steady_clock::now();
            try {
                run_step(e, dt_probe, opts, nullptr, st.data());
            } catch (const std::exception&) {
                return set_last_error(BO_ERR_STATE, "bo_ensemble_autotune: out of host memory");
            }
            const double sec =
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (seconds) seconds[order * ncand + c] = sec;
            for (int q = 0; q < count; ++q) {
                bo_status s = restore(e->members[q], snap[q]);
                if (s != BO_OK) return s;
            }
            bool ok = true;
            for (int q = 0; q < count; ++q) ok = ok && st[q] == BO_OK;
            if (ok && sec < best) {
                best = sec;
                best_w = candidates[c];
                best_lf = order == 0;
            }
        }
    }
    e->active = best_w;
    e->largest_first = best_lf;
    if (best < 1e300) return BO_OK;
    return set_last_error(BO_ERR_NOT_CONVERGED,
                          "bo_ensemble_autotune: no candidate schedule stepped every member");
}

bo_status bo_ensemble_autotune_precond(bo_ensemble* e, double dt_probe, const bo_newton_opts* opts,
                                      double* seconds, int* small_kind, int* large_kind) {
    if (e == nullptr || !(dt_probe > 0.0))
        return set_last_error(BO_ERR_INVALID_ARG,
                              "bo_ensemble_autotune_precond: NULL ensemble or dt_probe <= 0");
    const int count = (int)e->members.size();
    // size classes: members up to the median cell count, and the larger ones
    std::vector<int> sizes(count);
    for (int q = 0; q < count; ++q) sizes[q] = e->members[q]->geo.n;
    std::vector<int> sorted = sizes;
    std::sort(sorted.begin(), sorted.end());
    const int median = sorted[(count - 1) / 2];
    std::vector<Snapshot> snap(count);
    std::vector<int> kind0(count);
    for (int q = 0; q < count; ++q) {
        bo_status s = snapshot(e->members[q], snap[q]);
        if (s != BO_OK) return s;
        bo_get_preconditioner(e->members[q], &kind0[q]);
    }
    auto apply = [&](int ks, int kl) -> bo_status {
        for (int q = 0; q < count; ++q) {
            const bo_status s = bo_set_preconditioner(e->members[q], sizes[q] <= median ? ks : kl);
            if (s != BO_OK) return s;
        }
        return BO_OK;
    };
    const int combos[4][2] = {{BO_PRECOND_ILU0, BO_PRECOND_ILU0}, {BO_PRECOND_ILU0, BO_PRECOND_CPR},
                              {BO_PRECOND_CPR, BO_PRECOND_ILU0}, {BO_PRECOND_CPR, BO_PRECOND_CPR}};
    double best = 1e300;
    int best_c = -1;
    for (int c = 0; c < 4; ++c) {
        bo_status s = apply(combos[c][0], combos[c][1]);
        if (s != BO_OK) return s;
        std::vector<bo_status> st(count, BO_OK);
        const auto t0 = std::chrono::steady_clock::now();
        try {
            run_step(e, dt_probe, opts, nullptr, st.data());
        } catch (const std::exception&) {
            return set_last_error(BO_ERR_STATE, "bo_ensemble_autotune_precond: out of host memory");
        }
        const double sec =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (seconds) seconds[c] = sec;
        for (int q = 0; q < count; ++q) {
            s = restore(e->members[q], snap[q]);
            if (s != BO_OK) return s;
        }
        bool ok = true;
        for (int q = 0; q < count; ++q) ok = ok && st[q] == BO_OK;
        if (ok && sec < best) {
            best = sec;
            best_c = c;
        }
    }
    if (best_c < 0) {   // no combination stepped every member: back to what they had
        for (int q = 0; q < count; ++q) bo_set_preconditioner(e->members[q], kind0[q]);
        return set_last_error(BO_ERR_NOT_CONVERGED,
                              "bo_ensemble_autotune_precond: no combination stepped every member");
    }
    bo_status s = apply(combos[best_c][0], combos[best_c][1]);
    if (s != BO_OK) return s;
    if (small_kind) *small_kind = combos[best_c][0];
    if (large_kind) *large_kind = combos[best_c][1];
    return BO_OK;
}

bo_status bo_ensemble_autotune_schedule(bo_ensemble* e, double dt_probe, const bo_newton_opts* opts,
                                       double* seconds, int* small_schedule, int* streams) {
    if (e == nullptr || !(dt_probe > 0.0))
        return set_last_error(BO_ERR_INVALID_ARG,
                              "bo_ensemble_autotune_schedule: NULL ensemble or dt_probe <= 0");
    const int count = (int)e->members.size();
    std::vector<int> sizes(count);
    for (int q = 0; q < count; ++q) sizes[q] = e->members[q]->geo.n;
    std::vector<int> sorted = sizes;
    std::sort(sorted.begin(), sorted.end());
    const int median = sorted[(count - 1) / 2];
    std::vector<Snapshot> snap(count);
    std::vector<int> sched0(count);
    for (int q = 0; q < count; ++q) {
        bo_status s = snapshot(e->members[q], snap[q]);
        if (s != BO_OK) return s;
        sched0[q] = e->members[q]->solve_schedule;
    }
    const int w0 = e->active;
    const int wide = std::min(256, std::max(w0, 4 * w0));
    // (schedule of the small members, workers)
    const int combos[4][2] = {{BO_SCHEDULE_TILED, w0}, {BO_SCHEDULE_BLOCK, w0},
                              {BO_SCHEDULE_TILED, wide}, {BO_SCHEDULE_BLOCK, wide}};
    auto apply = [&](int kind) {
        for (int q = 0; q < count; ++q)
            e->members[q]->solve_schedule = sizes[q] <= median ? kind : BO_SCHEDULE_TILED;
    };
    double best = 1e300;
    int best_c = -1;
    for (int c = 0; c < 4; ++c) {
        apply(combos[c][0]);
        e->active = combos[c][1];
        std::vector<bo_status> st(count, BO_OK);
        const auto t0 = std::chrono::steady_clock::now();
        try {
            run_step(e, dt_probe, opts, nullptr, st.data());
        } catch (const std::exception&) {
            e->active = w0;
            return set_last_error(BO_ERR_STATE, "bo_ensemble_autotune_schedule: out of host memory");
        }
        const double sec =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (seconds) seconds[c] = sec;
        for (int q = 0; q < count; ++q) {
            const bo_status s = restore(e->members[q], snap[q]);
            if (s != BO_OK) {
                e->active = w0;
                return s;
            }
        }
        bool ok = true;
        for (int q = 0; q < count; ++q) ok = ok && st[q] == BO_OK;
        if (ok && sec < best) {
            best = sec;
            best_c = c;
        }
    }
    if (best_c < 0) {   // no combination stepped every member: back to what they had
        for (int q = 0; q < count; ++q) e->members[q]->solve_schedule = sched0[q];
        e->active = w0;
        return set_last_error(BO_ERR_NOT_CONVERGED,
                              "bo_ensemble_autotune_schedule: no combination stepped every member");
    }
    apply(combos[best_c][0]);
    e->active = combos[best_c][1];
    if (small_schedule) *small_schedule = combos[best_c][0];
    if (streams) *streams = combos[best_c][1];
    return BO_OK;
}

bo_status bo_ensemble_last_step_ms(const bo_ensemble* e, double* ms) {
    if (e == nullptr || ms == nullptr)
        return set_last_error(BO_ERR_INVALID_ARG, "bo_ensemble_last_step_ms: NULL argument");
    *ms = e->last_ms;
    return BO_OK;
}

bo_status bo_ensemble_destroy(bo_ensemble* e) {
    if (e == nullptr) return set_last_error(BO_ERR_INVALID_ARG, "bo_ensemble_destroy: NULL ensemble");
    for (auto& s : e->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t ev : e->ev_done) cudaEventDestroy(ev);
    if (e->ev_start) cudaEventDestroy(e->ev_start);
    if (e->ev_end) cudaEventDestroy(e->ev_end);
    if (e->tstream) cudaStreamDestroy(e->tstream);
    delete e;
    return BO_OK;
}

}  // extern "C"
