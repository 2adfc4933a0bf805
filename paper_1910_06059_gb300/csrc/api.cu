// C ABI of the black-oil library: object lifetime, memory, state I/O, the
// system export used for checking, and the host Newton loop of bo_step
// (arXiv 1910.06059 Section 2.3: Newton-Raphson on Eq. linsystem with
// Appleyard chop, variable switching and time-step cutting).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace bo {

static thread_local std::string g_last_error;

void fail(bo_status st, const std::string& msg) { throw Error{st, msg}; }

bo_status set_last_error(bo_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
    if (e == cudaSuccess) return;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                    std::to_string(line) + ")";
    fail(e == cudaErrorMemoryAllocation ? BO_ERR_OOM : BO_ERR_CUDA, m);
}

template <class F>
static bo_status guarded(F&& f) {
    try {
        f();
        return BO_OK;
    } catch (const Error& e) {
        g_last_error = e.msg;
        return e.status;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return BO_ERR_CUDA;
    }
}

template <class T>
static void dalloc(T** p, size_t count) {
    BO_CUDA(cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1)));
}

static void need(bool cond, bo_status st, const char* msg) {
    if (!cond) fail(st, msg);
}


void upload_aos3(bo_sim* s, const double* host, double* dev) {
    int n = s->geo.n;
    std::vector<double> soa(3 * (size_t)n);
    for (int c = 0; c < n; ++c)
        for (int e = 0; e < 3; ++e) soa[(size_t)e * n + c] = host[3 * (size_t)c + e];
    BO_CUDA(cudaMemcpyAsync(dev, soa.data(), sizeof(double) * soa.size(), cudaMemcpyHostToDevice,
                            s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
}

void download_aos3(const bo_sim* s, const double* dev, double* host) {
    int n = s->geo.n;
    std::vector<double> soa(3 * (size_t)n);
    BO_CUDA(cudaMemcpyAsync(soa.data(), dev, sizeof(double) * soa.size(), cudaMemcpyDeviceToHost,
                            s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
    for (int c = 0; c < n; ++c)
        for (int e = 0; e < 3; ++e) host[3 * (size_t)c + e] = soa[(size_t)e * n + c];
}

static void free_all(bo_sim* s) {
    destroy_graphs(s);
    cpr_free(s);
    dd_free(s);
    learn_set_clear(s);
    void* ptrs[] = {s->d_dx, s->d_dy, s->d_dz, s->d_perm, s->d_poro, s->d_T, s->d_pv, s->d_depth,
                    s->d_p, s->d_sw, s->d_x, s->d_flag, s->d_bk, s->d_bkflag, s->d_A0,
                    s->d_props, s->d_R, s->d_A, s->d_P, s->d_yt, s->d_qt, s->d_order, s->d_face, s->d_cellcon, s->d_wells,
                    s->d_con_cell, s->d_con_wi, s->d_wB, s->d_wC, s->d_b, s->d_xs, s->d_r,
                    s->d_rh, s->d_pk, s->d_v, s->d_s, s->d_t, s->d_ph, s->d_sh, s->d_part,
                    s->d_ks, s->d_ns, s->d_sweep_sync, s->d_P32, s->d_r32, s->d_y32,
                    s->d_ml_theta, s->d_ml_grad, s->d_ml_m, s->d_ml_v, s->d_ml_wbf,
                    s->d_ml_feat, s->d_ml_featf, s->d_ml_cell, s->d_ml_part, s->d_ml_delta,
                    s->d_ml_u, s->d_ml_z0, s->d_ml_e, s->d_ml_dd, s->d_ml_scal, s->d_ml_count,
                    s->d_ml_samples, s->d_ml_W, s->d_wB4, s->d_wC4, s->d_wcorr};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (s->h_ns) cudaFreeHost(s->h_ns);
    if (s->h_ks) cudaFreeHost(s->h_ks);
}

static void sync(bo_sim* s) { BO_CUDA(cudaStreamSynchronize(s->stream)); }

static void read_status(bo_sim* s) {
    BO_CUDA(cudaMemcpyAsync(s->h_ns, s->d_ns, sizeof(NewtonStatus), cudaMemcpyDeviceToHost,
                            s->stream));
    sync(s);
}

// Assembly plus the dead-well fix-up (one more assembly when a rate well has
// no flowing connection), then the norms.
static void assemble_and_norms(bo_sim* s, double dt) {
    launch_assemble(s, dt);
    read_status(s);
    if (s->h_ns->dead_wells > 0) {
        launch_fix_dead_wells(s);
        launch_assemble(s, dt);
    }
    launch_norms(s, dt);
    read_status(s);
    s->assembled = true;
    s->factored = false;
    s->solved = false;
    s->dt_last = dt;
}

// Online training on the residuals the last solve stored: opts epochs of
// one Adam step per residual on this system.
static void learn_online_step(bo_sim* s) {
    int cnt = 0;
    BO_CUDA(cudaMemcpyAsync(&cnt, s->d_ml_count, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
    cnt = std::min(cnt, s->ml_cap);
    if (cnt <= 0) return;
    const auto t0 = std::chrono::steady_clock::now();
    const size_t N = 3 * (size_t)s->geo.n;
    double first = 0.0, last = 0.0;
    for (int ep = 0; ep < s->ml_epochs; ++ep)
        for (int j = 0; j < cnt; ++j) {
            const double L = learn_loss_grad(s, s->d_ml_samples + (size_t)j * N);
            if (ep == 0) first += L;
            if (ep == s->ml_epochs - 1) last += L;
            learn_adam(s, s->ml_lr);
            s->ml_steps += 1;
        }
    BO_CUDA(cudaStreamSynchronize(s->stream));
    if (s->ml_first_loss < 0.0) s->ml_first_loss = first / cnt;
    s->ml_last_loss = last / cnt;
    s->ml_systems += 1;
    s->ml_train_ms +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Offline set of the learned stage: free every kept system.
void learn_set_clear(bo_sim* s) {
    for (LearnSystem& q : s->ml_set) {
        void* ptrs[] = {q.A, q.P, q.featf, q.cell, q.r};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    }
    s->ml_set.clear();
}

// Keep the last solve's system and its first residuals for offline training
// (while the set has room; a failed allocation ends the collection).
static void learn_store_system(bo_sim* s) {
    if ((int)s->ml_set.size() >= s->ml_collect_max) return;
    int cnt = 0;
    BO_CUDA(cudaMemcpyAsync(&cnt, s->d_ml_count, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
    const int nr = std::min(cnt, s->ml_cap);
    if (nr <= 0) return;
    const size_t n = s->geo.n, NA = 63 * n, NP = 63 * ilu_storage(s), NR = (size_t)nr * 3 * n;
    LearnSystem q;
    bool ok = cudaMalloc(reinterpret_cast<void**>(&q.A), sizeof(double) * NA) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&q.P), sizeof(double) * NP) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&q.featf), sizeof(float) * 64 * n) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&q.cell), sizeof(float4) * n) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&q.r), sizeof(double) * NR) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();   // the device is full: keep what was collected
        void* ptrs[] = {q.A, q.P, q.featf, q.cell, q.r};
        for (void* p : ptrs)
            if (p) cudaFree(p);
        s->ml_collect_max = (int)s->ml_set.size();
        return;
    }
    q.nr = nr;
    BO_CUDA(cudaMemcpyAsync(q.A, s->d_A, sizeof(double) * NA, cudaMemcpyDeviceToDevice, s->stream));
    BO_CUDA(cudaMemcpyAsync(q.P, s->d_P, sizeof(double) * NP, cudaMemcpyDeviceToDevice, s->stream));
    BO_CUDA(cudaMemcpyAsync(q.featf, s->d_ml_featf, sizeof(float) * 64 * n, cudaMemcpyDeviceToDevice,
                            s->stream));
    BO_CUDA(cudaMemcpyAsync(q.cell, s->d_ml_cell, sizeof(float4) * n, cudaMemcpyDeviceToDevice,
                            s->stream));
    BO_CUDA(cudaMemcpyAsync(q.r, s->d_ml_samples, sizeof(double) * NR, cudaMemcpyDeviceToDevice,
                            s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
    s->ml_set.push_back(q);
}

// Linear solve of the last assembly; returns the LS_* status.
static void check_timeout(bo_sim* s) {
    if (sweep_timeout(s)) {
        // leave the face buffers and the flag ready for the next call
        reset_sweep_faces(s);
        BO_CUDA(cudaMemsetAsync(s->d_sweep_sync + 2, 0, sizeof(int), s->stream));
        sync(s);
        fail(BO_ERR_DEVICE_TIMEOUT,
             "a dataflow sweep gave up waiting for a neighbour (bounded wait ran out)");
    }
}

static int solve_linear(bo_sim* s, double tol, int maxit, int* its) {
    launch_factor(s);
    read_status(s);
    check_timeout(s);
    if (s->h_ns->pad != 0) {  // non-finite pivot block
        *its = 0;
        return LS_BREAKDOWN;
    }
    if (s->h_ns->singular_wells > 0) {   // a full standard well with a singular D_w
        *its = 0;
        return LS_BREAKDOWN;
    }
    if (s->precond == BO_PRECOND_CPR) {   // a singular pivot of the coarsest pressure operator
        int bad = 0;
        BO_CUDA(cudaMemcpy(&bad, cpr_status_ptr(s), sizeof(int), cudaMemcpyDeviceToHost));
        if (bad) {
            *its = 0;
            return LS_BREAKDOWN;
        }
    }
    s->factored = true;
    s->last_fallback = 0;
    int st = run_bicgstab(s, tol, maxit, its, true);
    check_timeout(s);
    if (st != LS_OK && s->ml_on) {
        // the learned stage failed on this system: repeat with plain ILU(0)
        s->ml_fallbacks += 1;
        s->last_fallback |= 1;
        int its2 = 0;
        st = run_bicgstab(s, tol, maxit, &its2, false);
        check_timeout(s);
        *its += its2;
    }
    if (st != LS_OK && s->mixed) {
        // the FP32 sweeps failed on this system: repeat with the FP64 factors
        // and sweeps (the factorisation is FP64 in both modes)
        s->last_fallback |= 2;
        fill_sweep_faces(s, false);
        int its3 = 0;
        st = run_bicgstab(s, tol, maxit, &its3, false, true);
        fill_sweep_faces(s, true);
        check_timeout(s);
        *its += its3;
    }
    if (st == LS_OK && s->ml_on && s->ml_guard_left > 0 && !(s->last_fallback & 1)) {
        // guard window: the same system with plain ILU(0); its solution is kept
        int its_plain = 0;
        const int st_plain = run_bicgstab(s, tol, maxit, &its_plain, false);
        check_timeout(s);
        s->ml_guard_stage_its += *its;
        s->ml_guard_plain_its += its_plain;
        *its += its_plain;
        if (st_plain == LS_OK) st = st_plain;
        if (--s->ml_guard_left == 0) {
            const bool keep = s->ml_guard_stage_its < s->ml_guard_plain_its;
            s->ml_guard_state = keep ? 2 : 3;
            if (!keep) {
                s->ml_on = false;
                build_graphs(s);
            }
        }
    }
    if (s->ml_online) learn_online_step(s);
    if (s->ml_collect_max > 0) learn_store_system(s);
    launch_well_recover(s);
    s->solved = true;
    return st;
}

static bool norms_converged(const double* nrm, const bo_newton_opts& o, bool* finite) {
    *finite = true;
    for (int q = 0; q < 7; ++q)
        if (!std::isfinite(nrm[q])) *finite = false;
    bool conv = true;
    for (int a = 0; a < 3; ++a)
        if (nrm[a] > o.tol_mb || nrm[3 + a] > o.tol_cnv) conv = false;
    if (nrm[6] > o.tol_well) conv = false;
    return conv;
}

// Sub-step growth after a converged Newton solve of nits iterations.
static double step_growth(int nits) {
    if (nits <= 4) return 2.0;
    if (nits <= 8) return 1.5;
    if (nits <= 12) return 1.0;
    return 0.7;
}

using clk = std::chrono::steady_clock;
static double ms_since(clk::time_point t0) {
    return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
}

// Newton solve of one sub-step; 0 converged, 1 max iterations, 2 non-finite
// norms, 3 linear breakdown.
static int newton(bo_sim* s, double dt, const bo_newton_opts& o, int* nits, int* lits,
                  bo_step_report* rep) {
    launch_begin_step(s);
    for (int it = 0;; ++it) {
        auto t0 = clk::now();
        assemble_and_norms(s, dt);
        rep->ms_assemble += ms_since(t0);
        const double* nrm = s->h_ns->norms;
        bool finite;
        bool conv = norms_converged(nrm, o, &finite);
        if (!finite) return 2;
        if (conv) {
            *nits = it;
            for (int a = 0; a < 3; ++a) {
                rep->mb[a] = nrm[a];
                rep->cnv[a] = nrm[3 + a];
            }
            rep->well_res = nrm[6];
            return 0;
        }
        if (it == o.max_newton) {
            *nits = it;
            return 1;
        }
        int li = 0;
        t0 = clk::now();
        int st = solve_linear(s, o.tol_lin, o.max_lin, &li);
        sync(s);
        rep->ms_solve += ms_since(t0);
        *lits += li;
        if (st != LS_OK) {  // breakdown or missed tolerance fails the Newton solve
            *nits = it + 1;
            return 3;
        }
        t0 = clk::now();
        launch_newton_update(s, o);
        rep->ms_update += ms_since(t0);
    }
}

}  // namespace bo

using namespace bo;

extern "C" {

const char* bo_last_error(void) { return g_last_error.c_str(); }

bo_status bo_create_grid(int nx, int ny, int nz, const double* dx, const double* dy,
                         const double* dz, double top_depth, bo_sim** out) {
    return guarded([&] {
        need(out != nullptr, BO_ERR_INVALID_ARG, "bo_create_grid: out is NULL");
        *out = nullptr;
        need(nx > 0 && ny > 0 && nz > 0, BO_ERR_INVALID_ARG, "bo_create_grid: grid sizes must be positive");
        need((long long)nx * ny * nz < (1LL << 30), BO_ERR_INVALID_ARG,
             "bo_create_grid: more than 2^30 cells");
        need(dx && dy && dz, BO_ERR_INVALID_ARG, "bo_create_grid: dx, dy, dz must be given");
        for (int i = 0; i < nx; ++i) need(dx[i] > 0, BO_ERR_INVALID_ARG, "bo_create_grid: dx must be > 0");
        for (int j = 0; j < ny; ++j) need(dy[j] > 0, BO_ERR_INVALID_ARG, "bo_create_grid: dy must be > 0");
        for (int k = 0; k < nz; ++k) need(dz[k] > 0, BO_ERR_INVALID_ARG, "bo_create_grid: dz must be > 0");
        bo_sim* s = new bo_sim();
        try {
            s->geo = {nx, ny, nz, nx * ny * nz};
            s->dx.assign(dx, dx + nx);
            s->dy.assign(dy, dy + ny);
            s->dz.assign(dz, dz + nz);
            s->top = top_depth;
            BO_CUDA(cudaGetDevice(&s->device));
            size_t n = s->geo.n;
            dalloc(&s->d_dx, nx);
            dalloc(&s->d_dy, ny);
            dalloc(&s->d_dz, nz);
            BO_CUDA(cudaMemcpy(s->d_dx, dx, sizeof(double) * nx, cudaMemcpyHostToDevice));
            BO_CUDA(cudaMemcpy(s->d_dy, dy, sizeof(double) * ny, cudaMemcpyHostToDevice));
            BO_CUDA(cudaMemcpy(s->d_dz, dz, sizeof(double) * nz, cudaMemcpyHostToDevice));
            dalloc(&s->d_perm, 3 * (size_t)n);
            dalloc(&s->d_poro, n);
            dalloc(&s->d_T, 3 * n);
            dalloc(&s->d_pv, n);
            dalloc(&s->d_depth, n);
            dalloc(&s->d_p, n);
            dalloc(&s->d_sw, n);
            dalloc(&s->d_x, n);
            dalloc(&s->d_flag, n);
            dalloc(&s->d_bk, 3 * n);
            dalloc(&s->d_bkflag, n);
            dalloc(&s->d_A0, 3 * n);
            dalloc(&s->d_props, (size_t)NPROP * n);
            dalloc(&s->d_R, 3 * n);
            dalloc(&s->d_A, 63 * n);
            dalloc(&s->d_P, 63 * ilu_storage(s));
            // idle slots of the tile order are never written: zero factors
            BO_CUDA(cudaMemset(s->d_P, 0, sizeof(double) * 63 * ilu_storage(s)));
            dalloc(&s->d_yt, 3 * ilu_storage(s));
            dalloc(&s->d_qt, 3 * ilu_storage(s));
            dalloc(&s->d_order, 2 * (size_t)tile_count(s));
            dalloc(&s->d_face, face_storage(s));
            dalloc(&s->d_sweep_sync, 4);
            for (double** v : {&s->d_b, &s->d_xs, &s->d_r, &s->d_rh, &s->d_pk, &s->d_v, &s->d_s,
                               &s->d_t, &s->d_ph, &s->d_sh})
                dalloc(v, 3 * n);
            BO_CUDA(cudaMemset(s->d_A, 0, sizeof(double) * 63 * n));
            BO_CUDA(cudaMemset(s->d_p, 0, sizeof(double) * n));
            BO_CUDA(cudaMemset(s->d_sw, 0, sizeof(double) * n));
            BO_CUDA(cudaMemset(s->d_x, 0, sizeof(double) * n));
            BO_CUDA(cudaMemset(s->d_flag, 0, n));
            dalloc(&s->d_ks, 1);
            dalloc(&s->d_ns, 1);
            BO_CUDA(cudaMemset(s->d_ns, 0, sizeof(NewtonStatus)));
            BO_CUDA(cudaMallocHost(reinterpret_cast<void**>(&s->h_ns), sizeof(NewtonStatus)));
            BO_CUDA(cudaMallocHost(reinterpret_cast<void**>(&s->h_ks), sizeof(KrylovScalars)));
            setup_sweeps(s);
        } catch (...) {
            free_all(s);
            delete s;
            throw;
        }
        *out = s;
    });
}

bo_status bo_set_properties(bo_sim* s, const double* perm, const double* poro,
                            const bo_fluid* fluid, const bo_well* wells, int nwells) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_set_properties: sim is NULL");
        need(perm && poro && fluid, BO_ERR_INVALID_ARG, "bo_set_properties: perm, poro, fluid required");
        need(nwells >= 0 && (nwells == 0 || wells), BO_ERR_INVALID_ARG, "bo_set_properties: bad wells");
        need(!s->props_set, BO_ERR_STATE, "bo_set_properties: properties already set");
        const int n = s->geo.n;
        for (size_t c = 0; c < 3 * (size_t)n; ++c)
            need(perm[c] > 0 && std::isfinite(perm[c]), BO_ERR_INVALID_ARG,
                 "bo_set_properties: perm must be > 0 and finite (3n values: kx, ky, kz)");
        for (int c = 0; c < n; ++c)
            need(poro[c] > 0 && poro[c] <= 1, BO_ERR_INVALID_ARG, "bo_set_properties: poro must be in (0, 1]");
        static_assert(sizeof(bo_fluid) == sizeof(DevFluid), "fluid layout");
        std::memcpy(&s->fluid, fluid, sizeof(DevFluid));
        // wells
        std::vector<int> cellcon(n, -1), conwell;
        std::vector<double> rw, skin;
        s->wells_h.clear();
        s->con_cell_h.clear();
        s->well_volume.clear();
        s->nrate = 0;
        for (int w = 0; w < nwells; ++w) {
            const bo_well& in = wells[w];
            need(in.kind == 0 || in.kind == 1, BO_ERR_INVALID_ARG, "well kind must be 0 or 1");
            need(in.control == 0 || in.control == 1, BO_ERR_INVALID_ARG, "well control must be 0 or 1");
            need(in.kind == 1 || in.phase == 0 || in.phase == 2, BO_ERR_INVALID_ARG,
                 "injector phase must be 0 (water) or 2 (gas)");
            need(in.ncon > 0 && in.cells, BO_ERR_INVALID_ARG, "well needs at least one connection");
            need(in.rw > 0, BO_ERR_INVALID_ARG, "well radius must be > 0");
            WellDev d{};
            d.kind = in.kind;
            d.phase = in.kind == 0 ? in.phase : 1;
            d.ctl0 = d.ctl = in.control;
            d.off = (int)s->con_cell_h.size();
            d.ncon = in.ncon;
            d.target = in.target;
            d.limit = in.bhp_limit;
            d.bhp = in.control == 1 ? in.target : in.bhp_limit;
            if (in.control == 0) s->nrate++;
            for (int q = 0; q < in.ncon; ++q) {
                int c = in.cells[q];
                need(c >= 0 && c < n, BO_ERR_INVALID_ARG, "well connection cell out of range");
                need(cellcon[c] < 0, BO_ERR_INVALID_ARG, "a cell may hold only one well connection");
                cellcon[c] = (int)s->con_cell_h.size();
                s->con_cell_h.push_back(c);
                conwell.push_back(w);
            }
            // wellbore volume of the full standard well's storage term:
            // pi r_w^2 times the perforated thickness
            double thick = 0.0;
            for (int q = 0; q < in.ncon; ++q)
                thick += s->dz[in.cells[q] / (s->geo.nx * s->geo.ny)];
            s->well_volume.push_back(M_PI * in.rw * in.rw * thick);
            d.full = 0;
            d.vw = 0.0;
            rw.push_back(in.rw);
            skin.push_back(in.skin);
            s->wells_h.push_back(d);
        }
        s->nw = nwells;
        s->ncon = (int)s->con_cell_h.size();
        BO_CUDA(cudaMemcpy(s->d_perm, perm, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice));
        BO_CUDA(cudaMemcpy(s->d_poro, poro, sizeof(double) * n, cudaMemcpyHostToDevice));
        dalloc(&s->d_cellcon, (size_t)n + s->ncon);
        BO_CUDA(cudaMemcpy(s->d_cellcon, cellcon.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        if (s->ncon)
            BO_CUDA(cudaMemcpy(s->d_cellcon + n, conwell.data(), sizeof(int) * s->ncon,
                               cudaMemcpyHostToDevice));
        dalloc(&s->d_wells, s->nw);
        if (s->nw)
            BO_CUDA(cudaMemcpy(s->d_wells, s->wells_h.data(), sizeof(WellDev) * s->nw,
                               cudaMemcpyHostToDevice));
        dalloc(&s->d_con_cell, s->ncon);
        dalloc(&s->d_con_wi, s->ncon);
        dalloc(&s->d_wB, 3 * (size_t)s->ncon);
        dalloc(&s->d_wC, 3 * (size_t)s->ncon);
        if (s->ncon) {
            BO_CUDA(cudaMemcpy(s->d_con_cell, s->con_cell_h.data(), sizeof(int) * s->ncon,
                               cudaMemcpyHostToDevice));
            BO_CUDA(cudaMemset(s->d_wB, 0, sizeof(double) * 3 * s->ncon));
            BO_CUDA(cudaMemset(s->d_wC, 0, sizeof(double) * 3 * s->ncon));
        }
        // reduction scratch: props 1/b partials + norm partials, or Krylov partials + well scalars
        size_t npart = std::max<size_t>(3 * (size_t)props_blocks(s) + 7 * 1024,
                                        8 * (size_t)(152 * 4) + s->nw + 1);
        dalloc(&s->d_part, npart);
        double *d_rw = nullptr, *d_skin = nullptr;
        dalloc(&d_rw, s->nw);
        dalloc(&d_skin, s->nw);
        if (s->nw) {
            BO_CUDA(cudaMemcpy(d_rw, rw.data(), sizeof(double) * s->nw, cudaMemcpyHostToDevice));
            BO_CUDA(cudaMemcpy(d_skin, skin.data(), sizeof(double) * s->nw, cudaMemcpyHostToDevice));
        }
        launch_static(s);
        launch_wi(s, s->d_cellcon + n, d_rw, d_skin);
        sync(s);
        cudaFree(d_rw);
        cudaFree(d_skin);
        build_graphs(s);
        s->props_set = true;
    });
}

bo_status bo_get_static(const bo_sim* s, double* Tx, double* Ty, double* Tz, double* pv,
                        double* depth, double* wi) {
    return guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_get_static: properties not set");
        size_t n = s->geo.n;
        if (Tx) BO_CUDA(cudaMemcpy(Tx, s->d_T, sizeof(double) * n, cudaMemcpyDeviceToHost));
        if (Ty) BO_CUDA(cudaMemcpy(Ty, s->d_T + n, sizeof(double) * n, cudaMemcpyDeviceToHost));
        if (Tz) BO_CUDA(cudaMemcpy(Tz, s->d_T + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToHost));
        if (pv) BO_CUDA(cudaMemcpy(pv, s->d_pv, sizeof(double) * n, cudaMemcpyDeviceToHost));
        if (depth) BO_CUDA(cudaMemcpy(depth, s->d_depth, sizeof(double) * n, cudaMemcpyDeviceToHost));
        if (wi && s->ncon)
            BO_CUDA(cudaMemcpy(wi, s->d_con_wi, sizeof(double) * s->ncon, cudaMemcpyDeviceToHost));
    });
}

// Well start-up after an initial state: BHP wells at their target, rate wells
// first at their limit, then a rate-controlled injector at the BHP that meets
// its target by the linear inflow relation of the initial state.
static void start_wells(bo_sim* s) {
    for (auto& w : s->wells_h) w.bhp = w.ctl0 == 1 ? w.target : w.limit;
    for (int w = 0; w < s->nw; ++w) {
        WellDev d = s->wells_h[w];
        d.ctl = d.ctl0;
        BO_CUDA(cudaMemcpyAsync(s->d_wells + w, &d, sizeof(WellDev), cudaMemcpyHostToDevice,
                                s->stream));
        BO_CUDA(cudaStreamSynchronize(s->stream));
    }
    // datum densities at the initial state, then the injector BHP estimate
    launch_begin_step(s);
    launch_well_init_bhp(s);
    if (s->well_model == BO_WELL_MODEL_STANDARD) launch_std_wells_init(s);
    sync(s);
    s->assembled = s->factored = s->solved = false;
}

bo_status bo_init_hydrostatic(bo_sim* s, double p_top, double sw, double rgo) {
    return guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_init_hydrostatic: properties not set");
        need(p_top > 0 && sw >= 0 && sw <= 1 && rgo >= 0, BO_ERR_INVALID_ARG,
             "bo_init_hydrostatic: bad initial values");
        launch_hydrostatic(s, p_top, sw, rgo);
        start_wells(s);
    });
}

bo_status bo_init_equilibrium(bo_sim* s, const bo_equil* e) {
    return guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_init_equilibrium: properties not set");
        need(e != nullptr, BO_ERR_INVALID_ARG, "bo_init_equilibrium: NULL input");
        need(e->datum_pressure > 0 && e->goc_depth <= e->woc_depth && e->rgo >= 0 &&
                 e->swc >= 0 && e->swc < 1.0 - s->fluid.s_orw - s->fluid.s_org &&
                 std::isfinite(e->datum_depth) && std::isfinite(e->woc_depth) &&
                 std::isfinite(e->goc_depth),
             BO_ERR_INVALID_ARG, "bo_init_equilibrium: bad input (GOC above WOC, p > 0, "
                                 "0 <= swc < 1 - s_orw - s_org)");
        const EquilDev d{e->datum_depth, e->datum_pressure, e->woc_depth, e->goc_depth, e->rgo,
                         e->swc};
        launch_equilibrium(s, d);
        start_wells(s);
    });
}

static void set_bhp(bo_sim* s, const double* bhp, cudaMemcpyKind kind) {
    if (!bhp || s->nw == 0) return;
    std::vector<double> h(s->nw);
    if (kind == cudaMemcpyDeviceToHost) {
        BO_CUDA(cudaMemcpyAsync(h.data(), bhp, sizeof(double) * s->nw, cudaMemcpyDeviceToHost, s->stream));
        sync(s);
    } else {
        std::memcpy(h.data(), bhp, sizeof(double) * s->nw);
    }
    for (int w = 0; w < s->nw; ++w)
        BO_CUDA(cudaMemcpyAsync(&s->d_wells[w].bhp, &h[w], sizeof(double), cudaMemcpyHostToDevice,
                                s->stream));
    sync(s);
}

static void get_bhp(const bo_sim* s, double* bhp, bool dev) {
    if (!bhp || s->nw == 0) return;
    std::vector<WellDev> w(s->nw);
    BO_CUDA(cudaMemcpyAsync(w.data(), s->d_wells, sizeof(WellDev) * s->nw, cudaMemcpyDeviceToHost,
                            s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
    std::vector<double> h(s->nw);
    for (int q = 0; q < s->nw; ++q) h[q] = w[q].bhp;
    if (dev) {
        BO_CUDA(cudaMemcpyAsync(bhp, h.data(), sizeof(double) * s->nw, cudaMemcpyHostToDevice, s->stream));
        BO_CUDA(cudaStreamSynchronize(s->stream));
    } else {
        std::memcpy(bhp, h.data(), sizeof(double) * s->nw);
    }
}

static bo_status set_state_impl(bo_sim* s, const double* p, const double* sw, const double* x,
                                const unsigned char* flag, const double* bhp, bool dev) {
    return guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_set_state: properties not set");
        need(p && sw && x && flag, BO_ERR_INVALID_ARG, "bo_set_state: p, sw, x, flag required");
        need(s->nw == 0 || bhp, BO_ERR_INVALID_ARG, "bo_set_state: well_bhp required");
        size_t n = s->geo.n;
        cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        BO_CUDA(cudaMemcpyAsync(s->d_p, p, sizeof(double) * n, k, s->stream));
        BO_CUDA(cudaMemcpyAsync(s->d_sw, sw, sizeof(double) * n, k, s->stream));
        BO_CUDA(cudaMemcpyAsync(s->d_x, x, sizeof(double) * n, k, s->stream));
        BO_CUDA(cudaMemcpyAsync(s->d_flag, flag, n, k, s->stream));
        set_bhp(s, bhp, dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
        if (s->well_model == BO_WELL_MODEL_STANDARD) launch_std_wells_init(s);
        sync(s);
        s->assembled = s->factored = s->solved = false;
    });
}

static bo_status get_state_impl(const bo_sim* s, double* p, double* sw, double* x,
                                unsigned char* flag, double* bhp, bool dev) {
    return guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_get_state: properties not set");
        size_t n = s->geo.n;
        cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (p) BO_CUDA(cudaMemcpyAsync(p, s->d_p, sizeof(double) * n, k, s->stream));
        if (sw) BO_CUDA(cudaMemcpyAsync(sw, s->d_sw, sizeof(double) * n, k, s->stream));
        if (x) BO_CUDA(cudaMemcpyAsync(x, s->d_x, sizeof(double) * n, k, s->stream));
        if (flag) BO_CUDA(cudaMemcpyAsync(flag, s->d_flag, n, k, s->stream));
        get_bhp(s, bhp, dev);
        BO_CUDA(cudaStreamSynchronize(s->stream));
    });
}

bo_status bo_set_state(bo_sim* s, const double* p, const double* sw, const double* x,
                       const unsigned char* flag, const double* bhp) {
    return set_state_impl(s, p, sw, x, flag, bhp, false);
}
bo_status bo_set_state_dev(bo_sim* s, const double* p, const double* sw, const double* x,
                           const unsigned char* flag, const double* bhp) {
    return set_state_impl(s, p, sw, x, flag, bhp, true);
}
bo_status bo_get_state(const bo_sim* s, double* p, double* sw, double* x, unsigned char* flag,
                       double* bhp) {
    return get_state_impl(s, p, sw, x, flag, bhp, false);
}
bo_status bo_get_state_dev(const bo_sim* s, double* p, double* sw, double* x, unsigned char* flag,
                           double* bhp) {
    return get_state_impl(s, p, sw, x, flag, bhp, true);
}

bo_status bo_set_stream(bo_sim* s, void* stream) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_set_stream: sim is NULL");
        s->stream = static_cast<cudaStream_t>(stream);
    });
}

bo_status bo_begin_step(bo_sim* s) {
    return guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_begin_step: properties not set");
        launch_begin_step(s);
        sync(s);
    });
}

bo_status bo_assemble(bo_sim* s, double dt) {
    return guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_assemble: properties not set");
        need(dt > 0 && std::isfinite(dt), BO_ERR_INVALID_ARG, "bo_assemble: dt must be > 0");
        launch_assemble(s, dt);
        launch_norms(s, dt);
        read_status(s);
        s->assembled = true;
        s->factored = s->solved = false;
        s->dt_last = dt;
    });
}

bo_status bo_norms(bo_sim* s, double dt, double* out7) {
    return guarded([&] {
        need(s && s->assembled, BO_ERR_STATE, "bo_norms: no assembly");
        need(out7 != nullptr, BO_ERR_INVALID_ARG, "bo_norms: out is NULL");
        launch_norms(s, dt);
        read_status(s);
        std::memcpy(out7, s->h_ns->norms, sizeof(double) * 7);
    });
}

bo_status bo_get_system(const bo_sim* s, int* rowptr, int* colind, double* vals, double* res,
                        int* nnzb_out) {
    return guarded([&] {
        need(s && s->assembled, BO_ERR_STATE, "bo_get_system: no assembly");
        const Geom& g = s->geo;
        const int n = g.n;
        std::vector<double> A;
        if (vals) {
            A.resize(63 * (size_t)n);
            BO_CUDA(cudaMemcpy(A.data(), s->d_A, sizeof(double) * A.size(), cudaMemcpyDeviceToHost));
        }
        int q = 0;
        const int plane = g.nx * g.ny;
        if (rowptr) rowptr[0] = 0;
        for (int c = 0; c < n; ++c) {
            int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / plane;
            // ascending column order: -z, -y, -x, diag, +x, +y, +z
            const int order[7] = {NB_MZ, NB_MY, NB_MX, NB_DIAG, NB_PX, NB_PY, NB_PZ};
            const bool has[7] = {k > 0, j > 0, i > 0, true, i + 1 < g.nx, j + 1 < g.ny, k + 1 < g.nz};
            const int col[7] = {c - plane, c - g.nx, c - 1, c, c + 1, c + g.nx, c + plane};
            for (int t = 0; t < 7; ++t) {
                if (!has[t]) continue;
                if (colind) colind[q] = col[t];
                if (vals)
                    for (int e = 0; e < 9; ++e)
                        vals[9 * (size_t)q + e] = A[(size_t)(order[t] * 9 + e) * n + c];
                ++q;
            }
            if (rowptr) rowptr[c + 1] = q;
        }
        if (nnzb_out) *nnzb_out = q;
        if (res) download_aos3(s, s->d_R, res);
    });
}

bo_status bo_get_well_rates(const bo_sim* s, double* rates, double* bhp, int* control) {
    return guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_get_well_rates: properties not set");
        if (s->nw == 0) return;
        std::vector<WellDev> w(s->nw);
        BO_CUDA(cudaMemcpyAsync(w.data(), s->d_wells, sizeof(WellDev) * s->nw,
                                cudaMemcpyDeviceToHost, s->stream));
        BO_CUDA(cudaStreamSynchronize(s->stream));
        for (int q = 0; q < s->nw; ++q) {
            if (rates)
                for (int a = 0; a < 3; ++a) rates[3 * q + a] = w[q].qs[a];
            if (bhp) bhp[q] = w[q].bhp;
            if (control) control[q] = w[q].ctl;
        }
    });
}

bo_status bo_get_wells(const bo_sim* s, double* Rw, double* Dw, double* B, double* C, int* control) {
    return guarded([&] {
        need(s && s->assembled, BO_ERR_STATE, "bo_get_wells: no assembly");
        if (s->nw == 0) return;
        std::vector<WellDev> w(s->nw);
        BO_CUDA(cudaMemcpy(w.data(), s->d_wells, sizeof(WellDev) * s->nw, cudaMemcpyDeviceToHost));
        for (int q = 0; q < s->nw; ++q) {
            if (Rw) Rw[q] = w[q].Rw;
            if (Dw) Dw[q] = w[q].Dw;
            if (control) control[q] = w[q].ctl;
        }
        if (B) BO_CUDA(cudaMemcpy(B, s->d_wB, sizeof(double) * 3 * s->ncon, cudaMemcpyDeviceToHost));
        if (C) BO_CUDA(cudaMemcpy(C, s->d_wC, sizeof(double) * 3 * s->ncon, cudaMemcpyDeviceToHost));
    });
}

bo_status bo_factor(bo_sim* s, double* dinv) {
    return guarded([&] {
        need(s && s->assembled, BO_ERR_STATE, "bo_factor: no assembly");
        launch_factor(s);
        read_status(s);
        check_timeout(s);
        need(s->h_ns->pad == 0, BO_ERR_LINEAR_BREAKDOWN, "bo_factor: singular pivot block");
        s->factored = true;
        if (dinv) export_dinv(s, dinv);
    });
}

bo_status bo_precond_apply(bo_sim* s, const double* r, double* z) {
    return guarded([&] {
        need(s && s->factored, BO_ERR_STATE, "bo_precond_apply: no factorisation");
        need(r && z, BO_ERR_INVALID_ARG, "bo_precond_apply: r, z required");
        upload_aos3(s, r, s->d_b);
        launch_precond(s, s->d_b, s->d_t);
        download_aos3(s, s->d_t, z);
        check_timeout(s);
    });
}

bo_status bo_apply_op(bo_sim* s, const double* x, double* y) {
    return guarded([&] {
        need(s && s->assembled, BO_ERR_STATE, "bo_apply_op: no assembly");
        need(x && y, BO_ERR_INVALID_ARG, "bo_apply_op: x, y required");
        upload_aos3(s, x, s->d_b);
        launch_op(s, s->d_b, s->d_t);
        download_aos3(s, s->d_t, y);
    });
}

bo_status bo_solve(bo_sim* s, const bo_solve_opts* o, bo_solve_report* rep, double* sol) {
    return guarded([&] {
        need(s && s->assembled, BO_ERR_STATE, "bo_solve: no assembly");
        need(o && o->tol > 0 && o->max_it > 0, BO_ERR_INVALID_ARG, "bo_solve: bad options");
        int its = 0;
        int st = solve_linear(s, o->tol, o->max_it, &its);
        sync(s);
        if (rep) {
            rep->iterations = its;
            rep->status = st;
            rep->restarts = s->last_restarts;
            rep->rel_res = s->last_rel_res;
            rep->fallback = s->last_fallback;
        }
        if (sol) {
            download_aos3(s, s->d_xs, sol);
            std::vector<WellDev> w(s->nw);
            if (s->nw)
                BO_CUDA(cudaMemcpy(w.data(), s->d_wells, sizeof(WellDev) * s->nw, cudaMemcpyDeviceToHost));
            if (s->well_model == BO_WELL_MODEL_STANDARD) {
                for (int q = 0; q < s->nw; ++q)
                    for (int k = 0; k < 4; ++k) sol[3 * (size_t)s->geo.n + 4 * q + k] = w[q].dxs[k];
            } else {
                for (int q = 0; q < s->nw; ++q) sol[3 * (size_t)s->geo.n + q] = w[q].xw;
            }
        }
    });
}

bo_status bo_dd_solve(bo_sim* s, const bo_solve_opts* o, bo_solve_report* rep, double* sol) {
    return guarded([&] {
        need(s && s->assembled, BO_ERR_STATE, "bo_dd_solve: no assembly");
        need(o && o->tol > 0 && o->max_it > 0, BO_ERR_INVALID_ARG, "bo_dd_solve: bad options");
        need(s->ysub > 0 && s->zsub == 0, BO_ERR_STATE,
             "bo_dd_solve: the subdomains are y slabs: call bo_set_subdomains with ysub > 0, zsub = 0");
        need(!s->mixed && s->precond == BO_PRECOND_ILU0 && !s->ml_on &&
                 s->well_model == BO_WELL_MODEL_REDUCED,
             BO_ERR_STATE, "bo_dd_solve: needs FP64 ILU(0) sweeps, no learned stage, reduced wells");
        launch_factor(s);
        read_status(s);
        check_timeout(s);
        int its = 0, st = LS_BREAKDOWN;
        if (s->h_ns->pad == 0) {
            s->factored = true;
            st = dd_bicgstab(s, o->tol, o->max_it, &its);
            check_timeout(s);
            launch_well_recover(s);
            s->solved = true;
        }
        sync(s);
        if (rep) {
            std::memset(rep, 0, sizeof(*rep));
            rep->iterations = its;
            rep->status = st;
        }
        if (sol) {
            download_aos3(s, s->d_xs, sol);
            std::vector<WellDev> w(s->nw);
            if (s->nw)
                BO_CUDA(cudaMemcpy(w.data(), s->d_wells, sizeof(WellDev) * s->nw, cudaMemcpyDeviceToHost));
            for (int q = 0; q < s->nw; ++q) sol[3 * (size_t)s->geo.n + q] = w[q].xw;
        }
    });
}

bo_status bo_newton_update(bo_sim* s, const bo_newton_opts* o) {
    return guarded([&] {
        need(s && s->solved, BO_ERR_STATE, "bo_newton_update: no solution");
        need(o != nullptr, BO_ERR_INVALID_ARG, "bo_newton_update: opts is NULL");
        launch_newton_update(s, *o);
        sync(s);
        s->assembled = s->factored = s->solved = false;
    });
}

bo_status bo_step(bo_sim* s, double dt, const bo_newton_opts* o, bo_step_report* rep) {
    bo_step_report local{};
    bo_step_report* r = rep ? rep : &local;
    std::memset(r, 0, sizeof(*r));
    bo_status status = guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_step: properties not set");
        need(o != nullptr, BO_ERR_INVALID_ARG, "bo_step: opts is NULL");
        need(dt > 0 && std::isfinite(dt), BO_ERR_INVALID_ARG, "bo_step: dt must be > 0");
        double t = 0.0;
        if (s->dt_next <= 0.0) s->dt_next = (o->dt_init > 0.0) ? o->dt_init : dt;
        while (t < dt * (1.0 - 1e-12)) {
            double dts = std::min(s->dt_next, dt - t);
            int nits = 0, lits = 0;
            int st = newton(s, dts, *o, &nits, &lits, r);
            r->newton_its += nits;
            r->lin_its += lits;
            if (st == 0) {
                t += dts;
                r->substeps++;
                s->dt_next = std::min(dts * step_growth(nits), dt);
                continue;
            }
            launch_restore(s);
            sync(s);
            r->cuts++;
            s->dt_next = dts * o->cut_factor;
            if (r->cuts > o->max_cuts) {
                r->status = 1;
                fail(BO_ERR_NOT_CONVERGED, "bo_step: Newton did not converge after the allowed time-step cuts");
            }
        }
        s->assembled = s->factored = s->solved = false;
    });
    return status;
}

bo_status bo_get_step_control(const bo_sim* s, double* dt_next) {
    return guarded([&] {
        need(s && dt_next, BO_ERR_INVALID_ARG, "bo_get_step_control: NULL argument");
        *dt_next = s->dt_next;
    });
}

bo_status bo_set_step_control(bo_sim* s, double dt_next) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_set_step_control: sim is NULL");
        need(dt_next >= 0 && std::isfinite(dt_next), BO_ERR_INVALID_ARG,
             "bo_set_step_control: dt_next must be >= 0");
        s->dt_next = dt_next;
    });
}

bo_status bo_set_precision(bo_sim* s, int precision) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_set_precision: sim is NULL");
        need(precision == BO_PRECISION_FP64 || precision == BO_PRECISION_MIXED, BO_ERR_INVALID_ARG,
             "bo_set_precision: precision must be BO_PRECISION_FP64 or BO_PRECISION_MIXED");
        need(s->props_set, BO_ERR_STATE, "bo_set_precision: call bo_set_properties first");
        const bool mixed = precision == BO_PRECISION_MIXED;
        if (mixed == s->mixed) return;
        sync(s);
        if (mixed && s->d_P32 == nullptr) {
            dalloc(&s->d_P32, factors32_floats(s));
            dalloc(&s->d_r32, vec32_floats(s));
            dalloc(&s->d_y32, vec32_floats(s));
        }
        s->mixed = mixed;
        if (mixed) convert_factors32(s, s->stream);  // factors of an earlier bo_factor stay usable
        reset_sweep_faces(s);
        build_graphs(s);
        sync(s);
    });
}

bo_status bo_set_subdomains(bo_sim* s, int ysub, int zsub) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_set_subdomains: sim is NULL");
        need(ysub == 0 || (ysub > 0 && ysub % 8 == 0), BO_ERR_INVALID_ARG,
             "bo_set_subdomains: ysub must be 0 or a positive multiple of 8");
        need(zsub == 0 || (zsub > 0 && zsub % 4 == 0), BO_ERR_INVALID_ARG,
             "bo_set_subdomains: zsub must be 0 or a positive multiple of 4");
        need(s->props_set, BO_ERR_STATE, "bo_set_subdomains: call bo_set_properties first");
        if (ysub == s->ysub && zsub == s->zsub) return;
        sync(s);
        s->ysub = ysub;
        s->zsub = zsub;
        update_sweep_order(s);
        s->factored = false;   // the factors of the other partition are stale
        reset_sweep_faces(s);
        build_graphs(s);
        sync(s);
    });
}

bo_status bo_get_subdomains(const bo_sim* s, int* ysub, int* zsub) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_get_subdomains: sim is NULL");
        if (ysub) *ysub = s->ysub;
        if (zsub) *zsub = s->zsub;
    });
}

bo_status bo_get_precision(const bo_sim* s, int* precision) {
    return guarded([&] {
        need(s != nullptr && precision != nullptr, BO_ERR_INVALID_ARG,
             "bo_get_precision: NULL argument");
        *precision = s->mixed ? BO_PRECISION_MIXED : BO_PRECISION_FP64;
    });
}

// ---------------------------------------------------------------------------
// Learned preconditioner stage
// ---------------------------------------------------------------------------
bo_status bo_learn_set_params(bo_sim* s, const double* theta, int nparam) {
    return guarded([&] {
        need(s != nullptr && theta != nullptr, BO_ERR_INVALID_ARG, "bo_learn_set_params: NULL argument");
        need(nparam == BO_LEARN_NPARAM, BO_ERR_INVALID_ARG,
             "bo_learn_set_params: nparam must be BO_LEARN_NPARAM");
        need(s->props_set, BO_ERR_STATE, "bo_learn_set_params: call bo_set_properties first");
        for (int q = 0; q < nparam; ++q)
            need(std::isfinite(theta[q]), BO_ERR_INVALID_ARG, "bo_learn_set_params: non-finite value");
        sync(s);
        learn_setup(s);
        std::vector<float> f(theta, theta + nparam);
        learn_set_params(s, f.data());
        s->ml_params = true;
    });
}

bo_status bo_learn_get_params(bo_sim* s, double* theta, int nparam) {
    return guarded([&] {
        need(s != nullptr && theta != nullptr, BO_ERR_INVALID_ARG, "bo_learn_get_params: NULL argument");
        need(nparam == BO_LEARN_NPARAM, BO_ERR_INVALID_ARG,
             "bo_learn_get_params: nparam must be BO_LEARN_NPARAM");
        need(s->ml_params, BO_ERR_STATE, "bo_learn_get_params: no parameters set");
        std::vector<float> f(nparam);
        learn_get_params(s, f.data());
        for (int q = 0; q < nparam; ++q) theta[q] = f[q];
    });
}

bo_status bo_learn_set_engine(bo_sim* s, int engine) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_learn_set_engine: sim is NULL");
        need(engine == BO_LEARN_ENGINE_MMA_SYNC || engine == BO_LEARN_ENGINE_TCGEN05,
             BO_ERR_INVALID_ARG, "bo_learn_set_engine: engine must be BO_LEARN_ENGINE_*");
        if (engine == s->ml_engine) return;
        sync(s);
        s->ml_engine = engine;
        if (s->props_set) build_graphs(s);   // the factorisation graph runs the network
        if (s->ml_on && s->assembled) enqueue_learn_features(s, s->stream);
        sync(s);
    });
}

bo_status bo_learn_get_engine(const bo_sim* s, int* engine) {
    return guarded([&] {
        need(s != nullptr && engine != nullptr, BO_ERR_INVALID_ARG, "bo_learn_get_engine: NULL argument");
        *engine = s->ml_engine;
    });
}

bo_status bo_learn_enable(bo_sim* s, int on) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_learn_enable: sim is NULL");
        need(!on || s->ml_params, BO_ERR_STATE, "bo_learn_enable: no parameters set");
        if ((on != 0) == s->ml_on) return;
        sync(s);
        s->ml_on = on != 0;
        build_graphs(s);
        if (s->ml_on && s->assembled) enqueue_learn_features(s, s->stream);
        sync(s);
    });
}

bo_status bo_learn_online(bo_sim* s, const bo_learn_opts* o) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_learn_online: sim is NULL");
        sync(s);
        if (o == nullptr) {
            if (!s->ml_online) return;
            s->ml_online = false;
            build_graphs(s);
            return;
        }
        need(s->ml_params, BO_ERR_STATE, "bo_learn_online: no parameters set");
        need(o->samples >= 1 && o->samples <= 64 && o->epochs >= 1 && o->epochs <= 100 &&
                 o->lr > 0.0 && o->lr < 1.0,
             BO_ERR_INVALID_ARG, "bo_learn_online: samples 1..64, epochs 1..100, 0 < lr < 1");
        learn_setup_training(s);
        if (s->ml_cap != o->samples) {
            if (s->d_ml_samples) cudaFree(s->d_ml_samples);
            s->d_ml_samples = nullptr;
            dalloc(&s->d_ml_samples, (size_t)o->samples * 3 * s->geo.n);
            s->ml_cap = o->samples;
        }
        s->ml_epochs = o->epochs;
        s->ml_lr = o->lr;
        s->ml_online = true;
        build_graphs(s);
        if (s->assembled) enqueue_learn_features(s, s->stream);
        sync(s);
    });
}

bo_status bo_learn_collect(bo_sim* s, int max_systems, int samples) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_learn_collect: sim is NULL");
        need(max_systems >= 0 && samples >= 1 && samples <= 64, BO_ERR_INVALID_ARG,
             "bo_learn_collect: max_systems >= 0, samples 1..64");
        sync(s);
        if (max_systems == 0) {   // stop collecting, keep the set
            if (s->ml_collect_max == 0) return;
            s->ml_collect_max = 0;
            build_graphs(s);
            return;
        }
        need(s->ml_params, BO_ERR_STATE, "bo_learn_collect: no parameters set");
        need(!s->ml_online || s->ml_cap == samples, BO_ERR_STATE,
             "bo_learn_collect: online training keeps a different number of residuals");
        learn_set_clear(s);
        learn_setup_training(s);
        if (s->ml_cap != samples) {
            if (s->d_ml_samples) cudaFree(s->d_ml_samples);
            s->d_ml_samples = nullptr;
            dalloc(&s->d_ml_samples, (size_t)samples * 3 * s->geo.n);
            s->ml_cap = samples;
        }
        s->ml_collect_max = max_systems;
        build_graphs(s);
        if (s->assembled) enqueue_learn_features(s, s->stream);
        sync(s);
    });
}

bo_status bo_learn_set_info(const bo_sim* s, int* systems, int* residuals) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_learn_set_info: sim is NULL");
        int r = 0;
        for (const LearnSystem& q : s->ml_set) r += q.nr;
        if (systems) *systems = (int)s->ml_set.size();
        if (residuals) *residuals = r;
    });
}

bo_status bo_learn_train_offline(bo_sim* s, int epochs, double lr, double* first_loss,
                                 double* last_loss) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_learn_train_offline: sim is NULL");
        need(epochs >= 1 && epochs <= 1000 && lr > 0.0 && lr < 1.0, BO_ERR_INVALID_ARG,
             "bo_learn_train_offline: epochs 1..1000, 0 < lr < 1");
        need(s->ml_params && !s->ml_set.empty(), BO_ERR_STATE,
             "bo_learn_train_offline: no parameters or an empty set (bo_learn_collect)");
        need(!s->mixed && s->precond == BO_PRECOND_ILU0, BO_ERR_STATE,
             "bo_learn_train_offline: needs the FP64 ILU(0) preconditioner");
        learn_setup_training(s);
        const auto t0 = std::chrono::steady_clock::now();
        const size_t N = 3 * (size_t)s->geo.n;
        // each kept system's Jacobian, ILU(0) data, features and scalings take
        // the place of the current ones while its residuals are trained on
        struct Swap {
            bo_sim* s;
            double *A, *P;
            float* featf;
            float4* cell;
            ~Swap() {
                s->d_A = A;
                s->d_P = P;
                s->d_ml_featf = featf;
                s->d_ml_cell = cell;
            }
        } keep{s, s->d_A, s->d_P, s->d_ml_featf, s->d_ml_cell};
        double first = 0.0, last = 0.0;
        long long cnt = 0;
        for (int ep = 0; ep < epochs; ++ep) {
            for (const LearnSystem& q : s->ml_set) {
                s->d_A = q.A;
                s->d_P = q.P;
                s->d_ml_featf = q.featf;
                s->d_ml_cell = q.cell;
                for (int j = 0; j < q.nr; ++j) {
                    const double L = learn_loss_grad(s, q.r + (size_t)j * N);
                    if (ep == 0) first += L;
                    if (ep == epochs - 1) last += L;
                    if (ep == 0) ++cnt;
                    learn_adam(s, lr);
                    s->ml_steps += 1;
                }
            }
        }
        sync(s);
        check_timeout(s);
        s->ml_train_ms +=
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (first_loss) *first_loss = first / std::max<long long>(cnt, 1);
        if (last_loss) *last_loss = last / std::max<long long>(cnt, 1);
    });
}

bo_status bo_learn_guard(bo_sim* s, int probe) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_learn_guard: sim is NULL");
        need(probe >= 0, BO_ERR_INVALID_ARG, "bo_learn_guard: probe must be >= 0");
        need(probe == 0 || s->ml_on, BO_ERR_STATE, "bo_learn_guard: the stage is not on");
        s->ml_guard_left = probe;
        s->ml_guard_stage_its = s->ml_guard_plain_its = 0;
        s->ml_guard_state = probe > 0 ? 1 : 0;
    });
}

bo_status bo_learn_get_report(const bo_sim* s, bo_learn_report* r) {
    return guarded([&] {
        need(s != nullptr && r != nullptr, BO_ERR_INVALID_ARG, "bo_learn_get_report: NULL argument");
        r->systems = s->ml_systems;
        r->steps = s->ml_steps;
        r->fallbacks = s->ml_fallbacks;
        r->first_loss = s->ml_first_loss;
        r->last_loss = s->ml_last_loss;
        r->train_ms = s->ml_train_ms;
        r->guard_stage_its = s->ml_guard_stage_its;
        r->guard_plain_its = s->ml_guard_plain_its;
        r->guard_state = s->ml_guard_state;
    });
}

bo_status bo_learn_delta(bo_sim* s, const double* r, double* delta) {
    return guarded([&] {
        need(s != nullptr && r != nullptr && delta != nullptr, BO_ERR_INVALID_ARG,
             "bo_learn_delta: NULL argument");
        need(s->ml_params, BO_ERR_STATE, "bo_learn_delta: no parameters set");
        need(s->assembled && s->factored, BO_ERR_STATE, "bo_learn_delta: no factorisation");
        upload_aos3(s, r, s->d_b);
        enqueue_learn_features(s, s->stream);
        BO_CUDA(cudaMemsetAsync(s->d_t, 0, sizeof(double) * 3 * s->geo.n, s->stream));
        enqueue_learn_apply(s, s->stream, s->d_b, s->d_t, nullptr);
        download_aos3(s, s->d_t, delta);
    });
}

bo_status bo_learn_loss_grad(bo_sim* s, const double* r, double* loss, double* grad) {
    return guarded([&] {
        need(s != nullptr && r != nullptr, BO_ERR_INVALID_ARG, "bo_learn_loss_grad: NULL argument");
        need(s->ml_params, BO_ERR_STATE, "bo_learn_loss_grad: no parameters set");
        need(s->assembled && s->factored, BO_ERR_STATE, "bo_learn_loss_grad: no factorisation");
        learn_setup_training(s);
        upload_aos3(s, r, s->d_b);
        enqueue_learn_features(s, s->stream);
        learn_clear_grad(s);
        const double L = learn_loss_grad(s, s->d_b);
        check_timeout(s);
        if (loss) *loss = L;
        if (grad) {
            std::vector<float> g(BO_LEARN_NPARAM);
            learn_get_grad(s, g.data());
            for (int q = 0; q < BO_LEARN_NPARAM; ++q) grad[q] = g[q];
        }
        learn_clear_grad(s);
        sync(s);
    });
}

bo_status bo_set_timing(bo_sim* s, int enabled) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_set_timing: sim is NULL");
        s->timing = enabled != 0;
        for (int q = 0; q < MAX_TIMERS; ++q) {
            s->timer_ms[q] = 0.0;
            s->timer_n[q] = 0;
        }
    });
}

bo_status bo_get_timing(const bo_sim* s, int max, char (*names)[32], double* ms_total,
                        long long* launches, int* count) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_get_timing: sim is NULL");
        int k = std::min(max, s->ntimers);
        for (int q = 0; q < k; ++q) {
            if (names) {
                std::strncpy(names[q], s->timer_name[q].c_str(), 31);
                names[q][31] = 0;
            }
            if (ms_total) ms_total[q] = s->timer_ms[q];
            if (launches) launches[q] = s->timer_n[q];
        }
        if (count) *count = k;
    });
}

bo_status bo_set_preconditioner(bo_sim* s, int kind) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_set_preconditioner: sim is NULL");
        need(kind == BO_PRECOND_ILU0 || kind == BO_PRECOND_CPR, BO_ERR_INVALID_ARG,
             "bo_set_preconditioner: kind must be BO_PRECOND_ILU0 or BO_PRECOND_CPR");
        need(s->props_set, BO_ERR_STATE, "bo_set_preconditioner: call bo_set_properties first");
        if (kind == s->precond) return;
        sync(s);
        if (kind == BO_PRECOND_CPR) cpr_build(s);
        s->precond = kind;
        s->factored = false;
        build_graphs(s);
        sync(s);
    });
}

bo_status bo_get_preconditioner(const bo_sim* s, int* kind) {
    return guarded([&] {
        need(s != nullptr && kind != nullptr, BO_ERR_INVALID_ARG, "bo_get_preconditioner: NULL argument");
        *kind = s->precond;
    });
}

bo_status bo_set_solve_schedule(bo_sim* s, int kind) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_set_solve_schedule: sim is NULL");
        need(kind == BO_SCHEDULE_TILED || kind == BO_SCHEDULE_BLOCK, BO_ERR_INVALID_ARG,
             "bo_set_solve_schedule: kind must be BO_SCHEDULE_TILED or BO_SCHEDULE_BLOCK");
        s->solve_schedule = kind;
    });
}

bo_status bo_get_solve_schedule(const bo_sim* s, int* kind) {
    return guarded([&] {
        need(s != nullptr && kind != nullptr, BO_ERR_INVALID_ARG, "bo_get_solve_schedule: NULL argument");
        *kind = s->solve_schedule;
    });
}

bo_status bo_cpr_hierarchy(const bo_sim* s, int max_levels, int* nlevels, int* sizes, int* agg) {
    return guarded([&] {
        need(s != nullptr && nlevels != nullptr && sizes != nullptr, BO_ERR_INVALID_ARG,
             "bo_cpr_hierarchy: NULL argument");
        need(cpr_levels(s) > 0, BO_ERR_STATE, "bo_cpr_hierarchy: CPR has not been selected");
        const int L = cpr_levels(s);
        *nlevels = L;
        for (int l = 0; l < L && l < max_levels; ++l) sizes[l] = cpr_level_size(s, l);
        if (agg) {
            size_t off = 0;
            for (int l = 0; l + 1 < L; ++l) {
                const std::vector<int>& a = cpr_aggregation(s, l);
                std::memcpy(agg + off, a.data(), sizeof(int) * a.size());
                off += a.size();
            }
        }
    });
}

bo_status bo_cpr_pressure_system(bo_sim* s, double* w, double* ap) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_cpr_pressure_system: sim is NULL");
        need(s->precond == BO_PRECOND_CPR && s->factored, BO_ERR_STATE,
             "bo_cpr_pressure_system: no factorisation with CPR selected");
        sync(s);
        cpr_export_pressure(s, w, ap);
    });
}

bo_status bo_cpr_vcycle(bo_sim* s, const double* b, double* x) {
    return guarded([&] {
        need(s != nullptr && b != nullptr && x != nullptr, BO_ERR_INVALID_ARG,
             "bo_cpr_vcycle: NULL argument");
        need(s->precond == BO_PRECOND_CPR && s->factored, BO_ERR_STATE,
             "bo_cpr_vcycle: no factorisation with CPR selected");
        cpr_vcycle_host(s, b, x);
    });
}

bo_status bo_set_sweep_ctas_per_sm(bo_sim* s, int k) {
    return guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_set_sweep_ctas_per_sm: call bo_set_properties first");
        need(k == 1 || k == 2, BO_ERR_INVALID_ARG, "bo_set_sweep_ctas_per_sm: k must be 1 or 2");
        if (k == s->sweep_ctas_per_sm) return;
        sync(s);
        s->sweep_ctas_per_sm = k;
        setup_sweeps64(s);   // residency check and tile lists for the new grid
        build_graphs(s);     // the captured launches carry the grid
    });
}

bo_status bo_set_well_model(bo_sim* s, int model, int storage) {
    return guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_set_well_model: call bo_set_properties first");
        need(model == BO_WELL_REDUCED || model == BO_WELL_STANDARD, BO_ERR_INVALID_ARG,
             "bo_set_well_model: model must be BO_WELL_REDUCED or BO_WELL_STANDARD");
        const bool full = model == BO_WELL_STANDARD;
        if (full) std_wells_setup(s);
        std::vector<WellDev> w(s->nw);
        if (s->nw) {
            BO_CUDA(cudaMemcpy(w.data(), s->d_wells, sizeof(WellDev) * s->nw, cudaMemcpyDeviceToHost));
            for (int q = 0; q < s->nw; ++q) {
                // the host mirror too: start_wells uploads it after an initial state
                w[q].full = s->wells_h[q].full = full ? 1 : 0;
                w[q].vw = s->wells_h[q].vw = (full && storage) ? s->well_volume[q] : 0.0;
            }
            BO_CUDA(cudaMemcpy(s->d_wells, w.data(), sizeof(WellDev) * s->nw, cudaMemcpyHostToDevice));
        }
        s->well_model = full ? BO_WELL_MODEL_STANDARD : BO_WELL_MODEL_REDUCED;
        s->well_storage = storage != 0;
        s->assembled = s->factored = s->solved = false;
        build_graphs(s);   // the operator's well part differs between the models
    });
}

bo_status bo_get_well_model(const bo_sim* s, int* model) {
    return guarded([&] {
        need(s != nullptr && model != nullptr, BO_ERR_INVALID_ARG,
             "bo_get_well_model: NULL argument");
        *model = s->well_model == BO_WELL_MODEL_STANDARD ? BO_WELL_STANDARD : BO_WELL_REDUCED;
    });
}

bo_status bo_get_std_wells(const bo_sim* s, double* B, double* C, double* D, double* Rw,
                           double* xw) {
    return guarded([&] {
        need(s && s->props_set, BO_ERR_STATE, "bo_get_std_wells: properties not set");
        need(s->well_model == BO_WELL_MODEL_STANDARD, BO_ERR_STATE,
             "bo_get_std_wells: the full standard well model is not selected");
        need(!(B || C || D || Rw) || s->assembled, BO_ERR_STATE, "bo_get_std_wells: no assembly");
        if (s->nw == 0) return;
        std::vector<WellDev> w(s->nw);
        BO_CUDA(cudaMemcpy(w.data(), s->d_wells, sizeof(WellDev) * s->nw, cudaMemcpyDeviceToHost));
        for (int q = 0; q < s->nw; ++q) {
            if (D) std::memcpy(D + 16 * (size_t)q, w[q].D, sizeof(double) * 16);
            if (Rw) std::memcpy(Rw + 4 * (size_t)q, w[q].Rs, sizeof(double) * 4);
            if (xw) std::memcpy(xw + 4 * (size_t)q, w[q].xs, sizeof(double) * 4);
        }
        if (B) BO_CUDA(cudaMemcpy(B, s->d_wB4, sizeof(double) * 12 * s->ncon, cudaMemcpyDeviceToHost));
        if (C) BO_CUDA(cudaMemcpy(C, s->d_wC4, sizeof(double) * 12 * s->ncon, cudaMemcpyDeviceToHost));
    });
}

bo_status bo_get_launch_count(const bo_sim* s, long long* count) {
    return guarded([&] {
        need(s != nullptr && count != nullptr, BO_ERR_INVALID_ARG,
             "bo_get_launch_count: NULL argument");
        *count = s->launches;
    });
}

bo_status bo_selftest_bounded_wait(bo_sim* s, double* seconds) {
    bo_status st = guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_selftest_bounded_wait: sim is NULL");
        double t = wait_selftest(s);
        if (seconds) *seconds = t;
    });
    if (st != BO_OK) return st;
    g_last_error = "bounded-wait self-test: the wait ran out and was reported";
    return BO_ERR_DEVICE_TIMEOUT;
}

bo_status bo_residual_norms_noalloc(const double* R, const double* pv, const double* b, int n,
                                    double dt, double* out6, void* stream) {
    return guarded([&] {
        residual_norms_noalloc(R, pv, b, n, dt, out6, static_cast<cudaStream_t>(stream));
    });
}

bo_status bo_sizes(const bo_sim* s, int* n, int* nwells, int* ncon, int* nnzb) {
    return guarded([&] {
        need(s != nullptr, BO_ERR_INVALID_ARG, "bo_sizes: sim is NULL");
        const Geom& g = s->geo;
        if (n) *n = g.n;
        if (nwells) *nwells = s->nw;
        if (ncon) *ncon = s->ncon;
        if (nnzb) {
            long long F = (long long)(g.nx - 1) * g.ny * g.nz + (long long)g.nx * (g.ny - 1) * g.nz +
                          (long long)g.nx * g.ny * (g.nz - 1);
            *nnzb = (int)(g.n + 2 * F);
        }
    });
}

bo_status bo_destroy(bo_sim* s) {
    return guarded([&] {
        if (!s) return;
        cudaStreamSynchronize(s->stream);
        free_all(s);
        delete s;
    });
}

}  // extern "C"
