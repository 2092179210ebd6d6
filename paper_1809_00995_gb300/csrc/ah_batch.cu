// ah_batch.cu -- batched ensembles and the continuous-batching server (host side).
//
// Both run many independent FP32 lattices (the paper's ensemble of runs with
// different seeds, eras and s, Sec. 4 and Table 3) on one GPU with the batched
// fused step of k_fused.cu: one persistent launch per step advances every
// resident lattice, whatever its size, by one leapfrog step (Eqs. up_pi, up_E,
// up_phi, up_A), each with its own coefficient table and step counter in device
// memory.  Steps between diagnostic points are replayed from a CUDA graph.
//
//  * ah_batch_run: a fixed set of lattices, each run to its own tau_end, with
//    diagnostics at step 0, every diag_every steps and at the end.
//  * ah_server_*: requests arrive at any time; a scheduler thread admits them
//    while slots and an HBM budget allow, keeps all admitted lattices resident,
//    steps them together in rounds, and retires each at its tau_end with its
//    final observables and submit/done times.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/ah.h"
#include "ah_internal.cuh"
#include "trace.h"

using namespace ah;

namespace {

constexpr int kZChunk = 64;        // planes per work item
constexpr int kServerRound = 20;   // longest round of the server (admission latency bound)
constexpr int kMaxBatchN = 1290;   // largest lattice side with 32-bit site indices (1290^3 < 2^31)

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// One lattice of a batch or of the server.
struct Lat {
    ah_config cfg;
    int N = 0;
    long long nsites = 0;
    int nsteps = 0, step = 0, cur = 0;
    void *mem = nullptr;
    size_t bytes = 0;
    Fields<float> F{};
    KickCoef<float> *coefs = nullptr;
    // server bookkeeping
    uint64_t id = 0;
    double t_submit = 0.0;
};

size_t lattice_bytes(const ah_config &c)
{
    const size_t n = (size_t)c.N * c.N * c.N;
    return align256(host_state_bytes32(n)) + align256(sizeof(KickCoef<float>) * (size_t)host_run_steps(c));
}

// Allocate (stream-ordered), write the random-phase state and the coefficient table.
cudaError_t lat_setup(Lat &L, cudaStream_t st)
{
    L.N = L.cfg.N;
    L.nsites = (long long)L.N * L.N * L.N;
    L.nsteps = (int)host_run_steps(L.cfg);
    L.step = 0;
    L.cur = 0;
    L.bytes = lattice_bytes(L.cfg);
    cudaError_t e = cudaMallocAsync(&L.mem, L.bytes, st);
    if (e != cudaSuccess) {
        L.mem = nullptr;
        cudaGetLastError();                  // clear the refused allocation's error
        return e;
    }
    host_carve32(L.F, L.mem, (size_t)L.nsites);
    L.coefs = reinterpret_cast<KickCoef<float> *>(static_cast<char *>(L.mem) + align256(host_state_bytes32(L.nsites)));
    std::vector<KickCoef<float>> tab(std::max(1, L.nsteps));
    for (int n = 0; n < L.nsteps; ++n) tab[n] = host_kick_coef32(L.cfg, n);
    e = cudaMemsetAsync(L.mem, 0, host_state_bytes32(L.nsites), st);
    if (e == cudaSuccess) e = launch_init_phase<float>(L.F.phr[0], L.F.phi[0], L.N, L.cfg.seed, L.cfg.sigma, st);
    if (e == cudaSuccess && L.nsteps > 0)
        e = cudaMemcpyAsync(L.coefs, tab.data(), sizeof(KickCoef<float>) * L.nsteps, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // tab is host memory of this frame
    return e;
}

cudaError_t lat_reinit(Lat &L, cudaStream_t st)
{
    L.step = 0;
    L.cur = 0;
    cudaError_t e = cudaMemsetAsync(L.mem, 0, host_state_bytes32(L.nsites), st);
    if (e == cudaSuccess) e = launch_init_phase<float>(L.F.phr[0], L.F.phi[0], L.N, L.cfg.seed, L.cfg.sigma, st);
    return e;
}

View<float> lat_view(const Lat &L)
{
    View<float> v{};
    const int c = L.cur;
    v.phr = L.F.phr[c]; v.phi = L.F.phi[c];
    v.th1 = L.F.th[c][0]; v.th2 = L.F.th[c][1]; v.th3 = L.F.th[c][2];
    v.pir = L.F.pir; v.pii = L.F.pii;
    v.e1 = L.F.el[0]; v.e2 = L.F.el[1]; v.e3 = L.F.el[2];
    return v;
}

// Device tables and scratch of one batched run (grown on demand).
struct Engine {
    cudaStream_t st = nullptr;
    int num_sms = 0, shape = 0;
    BatchLattice *d_lat = nullptr;
    BatchState *d_state = nullptr;
    int2 *d_items = nullptr;
    int *d_nitems = nullptr;
    unsigned int *d_counter = nullptr;
    int cap_lat = 0;
    long long cap_items = 0;
    DiagPartial *d_partials = nullptr, *d_result = nullptr, *h_result = nullptr;
    int nparts = 0;                    // entries of d_partials before d_result
    DiagList list{};
    unsigned long long *h_count = nullptr;
    int diag_blocks = 0;
    // (shape, R, lattices loaded) -> R batched steps
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
    bool use_graph = true;
    long long launches = 0;
    int rounds = 0;

    cudaError_t init(bool graph)
    {
        use_graph = graph;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        diag_blocks = diag_grid_blocks(num_sms);
        // partials of the whole-lattice pass: the most CTAs that any accepted
        // lattice side needs (the z-chunk count of the pass depends on N, so the
        // largest N does not give the largest grid: 1024^3 takes more CTAs
        // than 1290^3)
        int max_ctas = 0;
        for (int n = 4; n <= kMaxBatchN; ++n) max_ctas = std::max(max_ctas, fused_diag_ctas(n));
        nparts = std::max(diag_blocks, max_ctas);
        list.capacity = 1 << 20;
        if (e == cudaSuccess) e = cudaMalloc(&d_partials, sizeof(DiagPartial) * (nparts + 1));
        if (e == cudaSuccess) e = cudaMalloc(&list.count, sizeof(unsigned long long) * (1 + list.capacity));
        if (e == cudaSuccess) e = cudaMallocHost(&h_result, sizeof(DiagPartial) + 64);
        if (e == cudaSuccess) e = cudaMalloc(&d_nitems, sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&d_counter, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned int), st);
        if (e != cudaSuccess) return e;
        d_result = d_partials + nparts;
        list.items = list.count + 1;
        h_count = reinterpret_cast<unsigned long long *>(h_result + 1);
        return cudaSuccess;
    }

    void clear_graphs()
    {
        for (auto &g : graphs) cudaGraphExecDestroy(g.second);
        graphs.clear();
    }

    void release()
    {
        if (st) cudaStreamSynchronize(st);
        clear_graphs();
        cudaFree(d_lat); cudaFree(d_state); cudaFree(d_items);
        cudaFree(d_nitems); cudaFree(d_counter); cudaFree(d_partials);
        if (list.count) cudaFree(list.count);
        if (h_result) cudaFreeHost(h_result);
        if (st) cudaStreamDestroy(st);
        *this = Engine();
    }

    // Upload descriptors, states and work items of the lattices (largest first).
    cudaError_t load(std::vector<Lat *> &lats)
    {
        const int n = (int)lats.size();
        std::vector<BatchLattice> bl(n);
        std::vector<BatchState> bs(n);
        std::vector<int2> items;
        std::vector<int> order(n);
        for (int i = 0; i < n; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lats[a]->N > lats[b]->N; });
        for (int i = 0; i < n; ++i) {
            const Lat &L = *lats[i];
            BatchLattice &B = bl[i];
            B.F = L.F;
            B.N = L.N;
            batch_tiles(shape, L.N, &B.tiles_x, &B.tiles_y);
            B.zc = std::min(L.N, kZChunk);
            B.nchunk = (L.N + B.zc - 1) / B.zc;
            B.nsteps = L.nsteps;
            B.coefs = L.coefs;
            bs[i].step = L.step;
            bs[i].cur = L.cur;
        }
        for (int i : order) {
            const int cnt = bl[i].tiles_x * bl[i].tiles_y * bl[i].nchunk;
            for (int k = 0; k < cnt; ++k) items.push_back(make_int2(i, k));
        }
        cudaError_t e = cudaSuccess;
        if (n > cap_lat) {
            cudaFree(d_lat); cudaFree(d_state);
            cap_lat = std::max(n, 2 * cap_lat);
            e = cudaMalloc(&d_lat, sizeof(BatchLattice) * cap_lat);
            if (e == cudaSuccess) e = cudaMalloc(&d_state, sizeof(BatchState) * cap_lat);
            clear_graphs();
        }
        if (e == cudaSuccess && (long long)items.size() > cap_items) {
            cudaFree(d_items);
            cap_items = std::max<long long>((long long)items.size(), 2 * cap_items);
            e = cudaMalloc(&d_items, sizeof(int2) * cap_items);
            clear_graphs();
        }
        const int ni = (int)items.size();
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(d_lat, bl.data(), sizeof(BatchLattice) * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(d_state, bs.data(), sizeof(BatchState) * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && ni) e = cudaMemcpyAsync(d_items, items.data(), sizeof(int2) * ni, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_nitems, &ni, sizeof(int), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host vectors above
        nlat_loaded = n;
        return e;
    }
    int nlat_loaded = 0;

    // R batched steps of every loaded lattice (graph replay when enabled).
    cudaError_t steps(int R)
    {
        TraceRange tr("batch steps");
        if (R <= 0) return cudaSuccess;
        launches += 2LL * R;
        ++rounds;
        if (!use_graph) {
            for (int r = 0; r < R; ++r) {
                cudaError_t e = launch_fused_batch(shape, d_lat, d_state, nlat_loaded, d_items, d_nitems, d_counter,
                                                   num_sms, st);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        }
        const auto key = std::make_tuple(shape, R, nlat_loaded);
        auto it = graphs.find(key);
        if (it == graphs.end()) {
            cudaGraph_t g;
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            for (int r = 0; r < R && e == cudaSuccess; ++r)
                e = launch_fused_batch(shape, d_lat, d_state, nlat_loaded, d_items, d_nitems, d_counter, num_sms, st);
            cudaError_t e2 = cudaStreamEndCapture(st, &g);
            if (e != cudaSuccess) return e;
            if (e2 != cudaSuccess) return e2;
            cudaGraphExec_t ex;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return e;
            it = graphs.emplace(key, ex).first;
        }
        return cudaGraphLaunch(it->second, st);
    }

    // Observables of one lattice at its current step (the whole-lattice pass on
    // the step's tile walk; everything in FP64 if the near-cut list overflows).
    ah_status diag(const Lat &L, ah_obs *out)
    {
        TraceRange tr("batch diagnostics");
        const View<float> v = lat_view(L);
        const Box b{ 0, 0, 0, L.N, L.N, L.N };
        const DiagCoef dc = host_diag_coef(L.cfg, L.step);
        cudaError_t e = launch_diag_whole<float>(v, L.N, dc, d_partials, nparts, d_result, list, diag_blocks, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_result, d_result, sizeof(DiagPartial), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_count, list.count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && *h_count > (unsigned long long)list.capacity) {
            e = launch_diag<float>(v, L.N, b, dc, d_partials, diag_blocks, d_result, list, true, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h_result, d_result, sizeof(DiagPartial), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
        if (e != cudaSuccess) return host_fail(AH_ERR_CUDA, cudaGetErrorString(e));
        host_fill_obs(L.cfg, L.step, L.nsites, *h_result, out);
        return AH_OK;
    }
};

// Steps to the next diagnostic point or the end of lattice L.
int steps_to_event(const Lat &L)
{
    int next = L.nsteps;
    if (L.cfg.diag_every > 0) next = std::min(next, (L.step / L.cfg.diag_every + 1) * L.cfg.diag_every);
    return next - L.step;
}

void advance_mirror(Lat &L, int R)
{
    const int d = std::min(R, L.nsteps - L.step);
    L.step += d;
    L.cur ^= (d & 1);
}

ah_status check_batch_cfg(const ah_config &c)
{
    if (c.precision != AH_FP32) return host_fail(AH_ERR_ARG, "batched lattices must be FP32 (precision AH_FP32)");
    if (c.diag_every < 0) return host_fail(AH_ERR_ARG, "diag_every must be >= 0");
    if (c.N > kMaxBatchN) return host_fail(AH_ERR_ARG, "batched lattices need N <= 1290 (32-bit site indices)");
    return host_validate(c);
}

}  // namespace

// ------------------------------------------------------------------ batch
extern "C" ah_status ah_batch_run(const ah_config *cfgs, int32_t count, int32_t flags, ah_obs *series,
                                  int64_t series_cap, int64_t *series_len, ah_batch_stats *stats)
{
    if (!cfgs || count < 1 || (series && (series_cap < 1 || !series_len)))
        return host_fail(AH_ERR_ARG, "ah_batch_run: bad arguments");
    if (flags & ~(AH_BATCH_AUTOTUNE | AH_BATCH_NO_GRAPH)) return host_fail(AH_ERR_ARG, "ah_batch_run: unknown flags");
    for (int i = 0; i < count; ++i) {
        ah_status st = check_batch_cfg(cfgs[i]);
        if (st != AH_OK) return st;
    }
    const double t0 = now_s();
    Engine eng;
    std::vector<Lat> lats(count);
    std::vector<Lat *> ptrs(count);
    auto cleanup = [&]() {
        if (eng.st) cudaStreamSynchronize(eng.st);
        for (auto &L : lats)
            if (L.mem) cudaFreeAsync(L.mem, eng.st);
        eng.release();
    };
    cudaError_t e = eng.init(!(flags & AH_BATCH_NO_GRAPH));
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        lats[i].cfg = cfgs[i];
        ptrs[i] = &lats[i];
        e = lat_setup(lats[i], eng.st);
    }
    if (e != cudaSuccess) {
        cleanup();
        return host_fail(e == cudaErrorMemoryAllocation ? AH_ERR_OOM : AH_ERR_CUDA, cudaGetErrorString(e));
    }
    // shape: the fastest over two timed steps of the whole batch (states restored after)
    int best = 0;
    if (flags & AH_BATCH_AUTOTUNE) {
        float best_ms = 0.0f;
        bool timed = false;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        for (int s = 0; s < batch_shape_count() && e == cudaSuccess; ++s) {
            bool ok = true;
            for (auto &L : lats) ok = ok && batch_shape_ok(s, L.N);
            if (!ok) continue;
            eng.shape = s;
            e = batch_shape_prepare(s, eng.num_sms, eng.st);
            if (e == cudaSuccess) e = eng.load(ptrs);
            if (e != cudaSuccess) break;
            eng.use_graph = false;
            e = eng.steps(1);
            if (e == cudaSuccess) e = cudaEventRecord(a, eng.st);
            if (e == cudaSuccess) e = eng.steps(2);
            if (e == cudaSuccess) e = cudaEventRecord(b, eng.st);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
            if (e == cudaSuccess && (!timed || ms < best_ms)) { best = s; best_ms = ms; timed = true; }
            for (auto &L : lats)
                if (e == cudaSuccess) e = lat_reinit(L, eng.st);
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        eng.use_graph = !(flags & AH_BATCH_NO_GRAPH);
        eng.launches = 0;
        eng.rounds = 0;
    }
    eng.shape = best;
    if (e == cudaSuccess) e = batch_shape_prepare(best, eng.num_sms, eng.st);
    if (e == cudaSuccess) e = eng.load(ptrs);
    if (e != cudaSuccess) {
        cleanup();
        return host_fail(AH_ERR_CUDA, cudaGetErrorString(e));
    }
    const double t_setup = now_s() - t0;
    ah_status st = AH_OK;
    auto record = [&](int i) {
        if (!series) return AH_OK;
        ah_obs o;
        ah_status s2 = eng.diag(lats[i], &o);
        if (s2 != AH_OK) return s2;
        if (series_len[i] < series_cap) series[(int64_t)i * series_cap + series_len[i]] = o;
        series_len[i] += 1;
        return AH_OK;
    };
    if (series)
        for (int i = 0; i < count; ++i) series_len[i] = 0;
    for (int i = 0; i < count && st == AH_OK; ++i) st = record(i);     // step 0
    const double t1 = now_s();
    double site_updates = 0.0;
    for (auto &L : lats) site_updates += (double)L.nsites * L.nsteps;
    while (st == AH_OK) {
        int R = INT32_MAX;
        for (auto &L : lats)
            if (L.step < L.nsteps) R = std::min(R, steps_to_event(L));
        if (R == INT32_MAX) break;
        e = eng.steps(R);
        if (e == cudaSuccess) e = cudaStreamSynchronize(eng.st);
        if (e != cudaSuccess) { st = host_fail(AH_ERR_CUDA, cudaGetErrorString(e)); break; }
        for (int i = 0; i < count && st == AH_OK; ++i) {
            Lat &L = lats[i];
            if (L.step >= L.nsteps) continue;
            advance_mirror(L, R);
            const bool due = L.step == L.nsteps || (L.cfg.diag_every > 0 && L.step % L.cfg.diag_every == 0);
            if (due) st = record(i);
        }
    }
    const double t2 = now_s();
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->seconds = t2 - t1;
        stats->setup_seconds = t_setup;
        stats->site_updates = site_updates;
        stats->sims_per_hour = stats->seconds > 0 ? count * 3600.0 / stats->seconds : 0.0;
        stats->shape = best;
        stats->rounds = eng.rounds;
        stats->launches = eng.launches;
    }
    cleanup();
    return st;
}

// ------------------------------------------------------------------ server
struct ah_server {
    size_t budget = 0, used = 0;
    int max_slots = 0;
    double t_origin = 0.0;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    uint64_t next_id = 1;
    std::deque<std::unique_ptr<Lat>> pending;
    std::vector<std::unique_ptr<Lat>> active;
    struct Result { int state; ah_obs obs; double t_submit, t_done; std::string err; };
    std::map<uint64_t, Result> results;     // state: 0 pending, 1 running, 2 done, 3 cancelled, 4 failed
    std::vector<uint64_t> cancel_running;
    ah_server_stats stats{};
    Engine eng;
    std::thread worker;
    int device = 0;
    // host-side fault injection for tests: after this many rounds the step call
    // reports a (fake) device error instead of launching (0: off); set from
    // AH_FAKE_DEVICE_FAILURE_AFTER_ROUNDS at creation
    long long fail_after_rounds = 0, rounds_done = 0;
    bool broken = false;      // the worker stopped after a device error

    void run();
};

namespace {
enum { RQ_PENDING = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_CANCELLED = 3, RQ_FAILED = 4 };
}

void ah_server::run()
{
    cudaSetDevice(device);
    std::vector<Lat *> loaded;
    bool dirty = true;
    // the device failed: every queued or running request fails with its error
    // (pollers see AH_ERR_CUDA instead of waiting) and the worker stops
    auto fail_all = [&](cudaError_t e) {
        std::lock_guard<std::mutex> lk(mu);
        const double t = now_s() - t_origin;
        auto mark = [&](uint64_t id) {
            Result &r = results[id];
            if (r.state == RQ_PENDING || r.state == RQ_RUNNING) {
                r.state = RQ_FAILED;
                r.err = cudaGetErrorString(e);
                r.t_done = t;
            }
        };
        for (auto &L : active) {
            mark(L->id);
            if (L->mem) cudaFreeAsync(L->mem, eng.st);
            used -= L->bytes;
        }
        active.clear();
        for (auto &L : pending) mark(L->id);
        pending.clear();
        stop = true;
        broken = true;
    };
    while (true) {
        std::vector<std::unique_ptr<Lat>> admit;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] { return stop || !pending.empty() || !active.empty(); });
            if (stop) break;
            // cancellations of running requests
            for (uint64_t id : cancel_running) {
                for (size_t i = 0; i < active.size(); ++i)
                    if (active[i]->id == id) {
                        cudaFreeAsync(active[i]->mem, eng.st);
                        used -= active[i]->bytes;
                        active.erase(active.begin() + i);
                        dirty = true;
                        break;
                    }
            }
            cancel_running.clear();
            // admission: FIFO while a slot and the budget allow
            while (!pending.empty() && (int)(active.size() + admit.size()) < max_slots &&
                   used + pending.front()->bytes <= budget) {
                used += pending.front()->bytes;
                results[pending.front()->id].state = RQ_RUNNING;
                admit.push_back(std::move(pending.front()));
                pending.pop_front();
            }
        }
        for (auto &L : admit) {
            const size_t bytes = L->bytes;
            const cudaError_t e = lat_setup(*L, eng.st);
            std::lock_guard<std::mutex> lk(mu);
            if (e != cudaSuccess) {
                used -= bytes;
                Result &r = results[L->id];
                r.state = RQ_FAILED;
                r.err = cudaGetErrorString(e);
                r.t_done = now_s() - t_origin;
                continue;
            }
            L->bytes = bytes;
            active.push_back(std::move(L));
            dirty = true;
            stats.admitted += 1;
        }
        if (active.empty()) continue;
        if (dirty) {
            loaded.clear();
            for (auto &L : active) loaded.push_back(L.get());
            const cudaError_t e = eng.load(loaded);
            if (e != cudaSuccess) { fail_all(e); break; }
            dirty = false;
        }
        int R = kServerRound;
        for (auto *L : loaded) R = std::min(R, steps_to_event(*L));
        cudaError_t e = fail_after_rounds > 0 && rounds_done >= fail_after_rounds ? cudaErrorLaunchFailure
                                                                                   : eng.steps(R);
        if (e == cudaSuccess) e = cudaStreamSynchronize(eng.st);
        if (e != cudaSuccess) { fail_all(e); break; }
        ++rounds_done;
        {
            std::lock_guard<std::mutex> lk(mu);
            for (auto *L : loaded) stats.site_updates += (double)L->nsites * std::min(R, L->nsteps - L->step);
            stats.launches = eng.launches;
        }
        for (auto *L : loaded) advance_mirror(*L, R);
        // retire finished lattices with their final observables
        for (size_t i = 0; i < active.size();) {
            Lat &L = *active[i];
            if (L.step < L.nsteps) { ++i; continue; }
            ah_obs o;
            const ah_status ds = eng.diag(L, &o);
            cudaFreeAsync(L.mem, eng.st);
            std::lock_guard<std::mutex> lk(mu);
            Result &r = results[L.id];
            if (r.state != RQ_CANCELLED) {          // a cancel that arrived during its last round wins
                r.state = ds == AH_OK || ds == AH_ERR_NONFINITE ? RQ_DONE : RQ_FAILED;
                r.obs = o;
                r.t_done = now_s() - t_origin;
            }
            used -= L.bytes;
            stats.completed += 1;
            active.erase(active.begin() + i);
            dirty = true;
        }
    }
}

extern "C" {

ah_status ah_server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t flags, ah_server **out)
{
    if (!out || hbm_budget_bytes == 0 || max_slots < 1 || (flags & ~AH_BATCH_NO_GRAPH))
        return host_fail(AH_ERR_ARG, "ah_server_create: bad arguments");
    *out = nullptr;
    ah_server *s = new (std::nothrow) ah_server();
    if (!s) return host_fail(AH_ERR_OOM, "host allocation failed");
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->t_origin = now_s();
    if (const char *f = std::getenv("AH_FAKE_DEVICE_FAILURE_AFTER_ROUNDS")) s->fail_after_rounds = std::atoll(f);
    cudaGetDevice(&s->device);
    cudaError_t e = s->eng.init(!(flags & AH_BATCH_NO_GRAPH));
    if (e == cudaSuccess) e = batch_shape_prepare(0, s->eng.num_sms, s->eng.st);
    if (e != cudaSuccess) {
        s->eng.release();
        delete s;
        return host_fail(AH_ERR_CUDA, cudaGetErrorString(e));
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return AH_OK;
}

ah_status ah_server_submit(ah_server *s, const ah_config *cfg, uint64_t *req_id)
{
    if (!s || !cfg || !req_id) return host_fail(AH_ERR_ARG, "ah_server_submit: null argument");
    ah_status st = check_batch_cfg(*cfg);
    if (st != AH_OK) return st;
    auto L = std::make_unique<Lat>();
    L->cfg = *cfg;
    L->bytes = lattice_bytes(*cfg);
    if (L->bytes > s->budget) return host_fail(AH_ERR_OOM, "request larger than the server's HBM budget");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->broken) return host_fail(AH_ERR_CUDA, "the server stopped after a device error");
    L->id = s->next_id++;
    L->t_submit = now_s() - s->t_origin;
    ah_server::Result r{};
    r.state = RQ_PENDING;
    r.t_submit = L->t_submit;
    s->results[L->id] = r;
    *req_id = L->id;
    s->pending.push_back(std::move(L));
    s->stats.submitted += 1;
    s->cv.notify_all();
    return AH_OK;
}

ah_status ah_server_poll(ah_server *s, uint64_t id, ah_obs *final_out, double *t_submit, double *t_done)
{
    if (!s) return host_fail(AH_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(id);
    if (it == s->results.end()) return host_fail(AH_ERR_NOTFOUND, "unknown request id");
    const ah_server::Result &r = it->second;
    if (t_submit) *t_submit = r.t_submit;
    switch (r.state) {
    case RQ_DONE:
        if (final_out) *final_out = r.obs;
        if (t_done) *t_done = r.t_done;
        return AH_OK;
    case RQ_CANCELLED: return host_fail(AH_ERR_CANCELLED, "request was cancelled");
    case RQ_FAILED: return host_fail(AH_ERR_CUDA, r.err.empty() ? "request failed" : r.err.c_str());
    default: return AH_ERR_BUSY;
    }
}

ah_status ah_server_cancel(ah_server *s, uint64_t id)
{
    if (!s) return host_fail(AH_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(id);
    if (it == s->results.end()) return host_fail(AH_ERR_NOTFOUND, "unknown request id");
    if (it->second.state == RQ_PENDING) {
        for (auto p = s->pending.begin(); p != s->pending.end(); ++p)
            if ((*p)->id == id) { s->pending.erase(p); break; }
    } else if (it->second.state == RQ_RUNNING) {
        s->cancel_running.push_back(id);
    } else {
        return AH_OK;
    }
    it->second.state = RQ_CANCELLED;
    s->cv.notify_all();
    return AH_OK;
}

ah_status ah_server_stats_get(ah_server *s, ah_server_stats *out)
{
    if (!s || !out) return host_fail(AH_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->running = (int32_t)s->active.size();
    out->queued = (int32_t)s->pending.size();
    out->hbm_used = (int64_t)s->used;
    return AH_OK;
}

void ah_server_destroy(ah_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (auto &L : s->active)
        if (L->mem) cudaFreeAsync(L->mem, s->eng.st);
    s->eng.release();
    delete s;
}

}  // extern "C"
