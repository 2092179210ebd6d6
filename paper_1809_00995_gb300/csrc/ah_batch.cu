// ah_batch.cu -- batched ensembles and the continuous-batching server (host side).
//
// Both run many independent FP32 lattices (the paper's ensemble of runs with
// different seeds, eras and s, Sec. 4 and Table 3) on one GPU with the batched
// fused step of k_fused.cu: one persistent launch per step advances every
// resident lattice, whatever its size, by one leapfrog step (Eqs. up_pi, up_E,
// up_phi, up_A), each with its own coefficient table and step counter in device
// memory.  With AH_BATCH_TWO_STEP the batched two-step pass of k_fused2.cu
// advances every lattice by two steps per launch (temporal blocking; a round
// with an odd number of steps ends with one single-step launch).  Steps
// between diagnostic points are replayed from a CUDA graph.
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
#include <cstdio>
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
constexpr int kZChunk2 = 256;      // planes per two-step work item (each also runs two extra planes)
// Two-step batches step the lattices of at least this side in pairs and the
// smaller ones one step per launch: the two-step tile writes 30 x 6 of its
// 32 x 8 sites, so small lattices pay more in partial tiles and halo
// recomputation than they save in DRAM traffic (on GB300 two-step passes tie
// single steps at 512^3 and win at 1024^3).
constexpr int kPairMinN = 512;
// Paired lattices of at least this side fill the GPU with their own two-step
// grid (512^3: 3096 CTAs): they run the single-lattice two-step kernel, whose
// pointers and coefficients are kernel parameters, instead of taking items of
// the persistent batched pass (which stages them in shared memory; 16.66
// against 15.47 ms per step at 1024^3).
constexpr int kDirectMinN = 512;
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
    int nsteps = 0, step = 0, cur = 0, pe = 0;
    bool two = false;                 // stepped in pairs (second Pi/E set for the two-step pass)
    bool weak = false;                // its last observables found max |theta| <= kWeakTheta (paired lattices)
    void *mem = nullptr;
    size_t bytes = 0;
    Fields<float> F{};
    KickCoef<float> *coefs = nullptr;
    // server bookkeeping
    uint64_t id = 0;
    double t_submit = 0.0;
    std::vector<ah_window> wins;      // windows written when the request completes
};

// A lattice is stepped in pairs if its configuration asks for it
// (AH_FLAG_TWO_STEP) or, with auto_pairs (AH_BATCH_TWO_STEP), if N >= kPairMinN.
bool lat_pairs(const ah_config &c, bool auto_pairs)
{
    return (c.flags & AH_FLAG_TWO_STEP) || (auto_pairs && c.N >= kPairMinN);
}

size_t lattice_bytes(const ah_config &c, bool two)
{
    const size_t n = (size_t)c.N * c.N * c.N;
    return align256(host_state_bytes32(n, two)) + align256(sizeof(KickCoef<float>) * (size_t)host_run_steps(c));
}

// Allocate (stream-ordered), write the random-phase state and the coefficient table.
cudaError_t lat_setup(Lat &L, bool two, cudaStream_t st)
{
    L.N = L.cfg.N;
    L.nsites = (long long)L.N * L.N * L.N;
    L.nsteps = (int)host_run_steps(L.cfg);
    L.step = 0;
    L.cur = 0;
    L.pe = 0;
    L.two = two;
    L.bytes = lattice_bytes(L.cfg, two);
    cudaError_t e = cudaMallocAsync(&L.mem, L.bytes, st);
    if (e != cudaSuccess) {
        L.mem = nullptr;
        cudaGetLastError();                  // clear the refused allocation's error
        return e;
    }
    const size_t sb = host_state_bytes32(L.nsites, two);
    host_carve32(L.F, L.mem, (size_t)L.nsites, two);
    L.coefs = reinterpret_cast<KickCoef<float> *>(static_cast<char *>(L.mem) + align256(sb));
    std::vector<KickCoef<float>> tab(std::max(1, L.nsteps));
    for (int n = 0; n < L.nsteps; ++n) tab[n] = host_kick_coef32(L.cfg, n);
    e = cudaMemsetAsync(L.mem, 0, sb, st);
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
    L.pe = 0;
    cudaError_t e = cudaMemsetAsync(L.mem, 0, host_state_bytes32(L.nsites, L.two), st);
    if (e == cudaSuccess) e = launch_init_phase<float>(L.F.phr[0], L.F.phi[0], L.N, L.cfg.seed, L.cfg.sigma, st);
    return e;
}

// The lattice's buffers with Pi and E of its current set in F.pir, F.pii, F.el.
Fields<float> lat_fields(const Lat &L)
{
    Fields<float> F = L.F;
    if (L.pe) {
        F.pir = L.F.spare[0];
        F.pii = L.F.spare[1];
        for (int d = 0; d < 3; ++d) F.el[d] = L.F.spare[2 + d];
    }
    return F;
}

View<float> lat_view(const Lat &L)
{
    const Fields<float> F = lat_fields(L);
    View<float> v{};
    const int c = L.cur;
    v.phr = F.phr[c]; v.phi = F.phi[c];
    v.th1 = F.th[c][0]; v.th2 = F.th[c][1]; v.th3 = F.th[c][2];
    v.pir = F.pir; v.pii = F.pii;
    v.e1 = F.el[0]; v.e2 = F.el[1]; v.e3 = F.el[2];
    return v;
}

ah_status check_window(const ah_window &w, int N)
{
    if (!w.out) return host_fail(AH_ERR_ARG, "window with a null output buffer");
    if (w.nx < 1 || w.ny < 1 || w.nz < 1 || w.nx > N || w.ny > N || w.nz > N)
        return host_fail(AH_ERR_ARG, "window extent must be in [1, N]");
    return AH_OK;
}

// Device tables and scratch of one batched run (grown on demand).
struct Engine {
    cudaStream_t st = nullptr;
    int num_sms = 0, shape = 0;
    bool two = false;                  // the batch may hold lattices stepped in pairs
    int shape2 = 0;                    // shape of the batched two-step pass
    BatchLattice *d_lat = nullptr;
    BatchState *d_state = nullptr;
    int2 *d_items = nullptr, *d_items2 = nullptr;
    int *d_nitems = nullptr;           // [0] single-step items, [1] two-step items
    unsigned int *d_counter = nullptr;
    int cap_lat = 0;
    long long cap_items = 0, cap_items2 = 0;
    DiagPartial *d_partials = nullptr, *d_result = nullptr, *h_result = nullptr;
    int nparts = 0;                    // entries of d_partials before d_result
    DiagList list{};
    unsigned long long *h_count = nullptr;
    int diag_blocks = 0;
    // (shape key, R, lattices loaded) -> R batched steps
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
    bool use_graph = true;
    long long launches = 0;
    long long weak_launches = 0;   // direct two-step launches in the form for weak gauge fields
    int rounds = 0;

    cudaError_t init(bool graph, bool two_step)
    {
        use_graph = graph;
        two = two_step;
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
        if (e == cudaSuccess) e = cudaMalloc(&d_nitems, 2 * sizeof(int));
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
        cudaFree(d_lat); cudaFree(d_state); cudaFree(d_items); cudaFree(d_items2);
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
        std::vector<int2> items, items2;
        std::vector<int> order(n);
        for (int i = 0; i < n; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lats[a]->N > lats[b]->N; });
        for (int i = 0; i < n; ++i) {
            const Lat &L = *lats[i];
            BatchLattice &B = bl[i];
            memset(&B, 0, sizeof B);
            B.F = L.F;
            float *const q0[5] = { L.F.pir, L.F.pii, L.F.el[0], L.F.el[1], L.F.el[2] };
            for (int k = 0; k < 5; ++k) {
                B.q[0][k] = q0[k];
                B.q[1][k] = L.F.spare[k];
            }
            B.N = L.N;
            batch_tiles(shape, L.N, &B.tiles_x, &B.tiles_y);
            B.zc = std::min(L.N, kZChunk);
            B.nchunk = (L.N + B.zc - 1) / B.zc;
            if (two && L.two) {
                B.pairs = 1;
                batch2_tiles(shape2, L.N, &B.tiles2_x, &B.tiles2_y);
                B.zc2 = std::min(L.N, kZChunk2);
                B.nchunk2 = (L.N + B.zc2 - 1) / B.zc2;
            }
            B.nsteps = L.nsteps;
            B.diag_every = L.cfg.diag_every;
            B.coefs = L.coefs;
            bs[i].step = L.step;
            bs[i].cur = L.cur;
            bs[i].pe = L.pe;
        }
        direct.clear();
        for (int i : order) {
            const int cnt = bl[i].tiles_x * bl[i].tiles_y * bl[i].nchunk;
            for (int k = 0; k < cnt; ++k) items.push_back(make_int2(i, k));
            if (bl[i].pairs && lats[i]->N >= kDirectMinN) {
                direct.push_back(lats[i]);           // its own grid launches, no items
                continue;
            }
            const int cnt2 = bl[i].tiles2_x * bl[i].tiles2_y * bl[i].nchunk2;
            for (int k = 0; k < cnt2; ++k) items2.push_back(make_int2(i, k));
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
        if (e == cudaSuccess && (long long)items2.size() > cap_items2) {
            cudaFree(d_items2);
            cap_items2 = std::max<long long>((long long)items2.size(), 2 * cap_items2);
            e = cudaMalloc(&d_items2, sizeof(int2) * cap_items2);
            clear_graphs();
        }
        const int ni[2] = { (int)items.size(), (int)items2.size() };
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(d_lat, bl.data(), sizeof(BatchLattice) * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(d_state, bs.data(), sizeof(BatchState) * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && ni[0])
            e = cudaMemcpyAsync(d_items, items.data(), sizeof(int2) * ni[0], cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && ni[1])
            e = cudaMemcpyAsync(d_items2, items2.data(), sizeof(int2) * ni[1], cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_nitems, ni, 2 * sizeof(int), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host vectors above
        nlat_loaded = n;
        n_paired = n_unpaired = 0;
        for (int i = 0; i < n; ++i) (bl[i].pairs ? n_paired : n_unpaired) += 1;
        return e;
    }
    int n_paired = 0, n_unpaired = 0;   // loaded lattices stepped in pairs / one step at a time
    std::vector<Lat *> direct;          // paired lattices run by the single-lattice two-step kernel

    // The two-step pass p of the current round of the directly launched lattice
    // L, from its host mirror (step, buffers, Pi/E set at the round's start).
    cudaError_t launch_direct(const Lat &L, int p)
    {
        const int n = L.step + 2 * p, cur = L.cur ^ (p & 1), pe = L.pe ^ (p & 1), o = 1 - cur;
        const Fields<float> &F = L.F;
        float *const q0[5] = { F.pir, F.pii, F.el[0], F.el[1], F.el[2] };
        float *const *q = pe ? F.spare : q0;
        float *const *oq = pe ? q0 : F.spare;
        View2<float> v;
        v.phr = F.phr[cur]; v.phi = F.phi[cur];
        v.th1 = F.th[cur][0]; v.th2 = F.th[cur][1]; v.th3 = F.th[cur][2];
        v.pir = q[0]; v.pii = q[1]; v.e1 = q[2]; v.e2 = q[3]; v.e3 = q[4];
        v.ophr = F.phr[o]; v.ophi = F.phi[o];
        v.oth1 = F.th[o][0]; v.oth2 = F.th[o][1]; v.oth3 = F.th[o][2];
        v.opir = oq[0]; v.opii = oq[1]; v.oe1 = oq[2]; v.oe2 = oq[3]; v.oe3 = oq[4];
        launches += 1;
        // the kernel for weak gauge fields while the lattice's last observables allow it
        const bool weak = L.weak && fused2_weak_ok(fused2_default_variant(), L.N);
        weak_launches += weak;
        return launch_fused2_step(v, L.N, host_kick_coef32(L.cfg, n), host_kick_coef32(L.cfg, n + 1),
                                  fused2_default_variant(), st, weak);
    }

    // The launches of a round of R batched steps (R: the fewest steps any
    // unfinished lattice has to its next stop).  One step per launch: R
    // launches.  Two-step mode: R / 2 times a two-step pass of the paired
    // lattices and two single steps of the others, then for an odd R one single
    // step of the others and of the paired lattices one step before their next
    // stop (the paired lattices keep their steps in pairs, see batch_stop).
    cudaError_t enqueue_steps(int R)
    {
        if (two) {
            auto single = [&](int mode) {
                launches += 2;
                return launch_fused_batch(shape, d_lat, d_state, nlat_loaded, d_items, d_nitems, d_counter, num_sms, st,
                                          mode);
            };
            for (int r = 0; r < R / 2; ++r) {
                for (const Lat *L : direct) {
                    // a lattice that has reached its end stays loaded until the
                    // batch is done: it takes no more passes (an unfinished one
                    // has at least R steps to its next stop and takes them all)
                    if (L->step >= L->nsteps) continue;
                    cudaError_t e = launch_direct(*L, r);
                    if (e != cudaSuccess) return e;
                }
                if (n_paired) {
                    // the other paired lattices; its advance kernel moves every
                    // paired lattice on, the directly launched ones included
                    cudaError_t e = launch_fused2_batch(shape2, d_lat, d_state, nlat_loaded, d_items2, d_nitems + 1,
                                                        d_counter, num_sms, st);
                    if (e != cudaSuccess) return e;
                    launches += 2;
                }
                for (int k = 0; k < 2 && n_unpaired; ++k) {
                    cudaError_t e = single(BATCH_UNPAIRED);
                    if (e != cudaSuccess) return e;
                }
            }
            if (R % 2) return single(BATCH_ROUND_END);
            return cudaSuccess;
        }
        for (int r = 0; r < R; ++r) {
            cudaError_t e = launch_fused_batch(shape, d_lat, d_state, nlat_loaded, d_items, d_nitems, d_counter,
                                               num_sms, st);
            if (e != cudaSuccess) return e;
            launches += 2;
        }
        return cudaSuccess;
    }
    int nlat_loaded = 0;

    // R batched steps of every loaded lattice (graph replay when enabled).
    cudaError_t steps(int R)
    {
        TraceRange tr("batch steps");
        if (R <= 0) return cudaSuccess;
        ++rounds;
        // a directly launched lattice takes its pointers and coefficients as
        // kernel parameters, which change from round to round: no graph then
        if (!use_graph || !direct.empty()) return enqueue_steps(R);
        const long long before = launches;
        const int mix = (n_paired ? 1 : 0) + (n_unpaired ? 2 : 0);
        const auto key = std::make_tuple(two ? 1000 + 64 * mix + 16 * shape2 + shape : shape, R, nlat_loaded);
        auto it = graphs.find(key);
        if (it == graphs.end()) {
            cudaGraph_t g;
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) e = enqueue_steps(R);
            cudaError_t e2 = cudaStreamEndCapture(st, &g);
            if (e != cudaSuccess) return e;
            if (e2 != cudaSuccess) return e2;
            cudaGraphExec_t ex;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return e;
            it = graphs.emplace(key, ex).first;
            launches = before;
        }
        launches = before + (two ? 2LL * ((R / 2) * ((n_paired ? 1 : 0) + (n_unpaired ? 2 : 0)) + R % 2)
                                 : 2LL * R);
        return cudaGraphLaunch(it->second, st);
    }

    // Copy window w of lattice L's current state to w.out (host, FP64).
    ah_status gather(const Lat &L, const ah_window &w)
    {
        const int N = L.N;
        auto md = [N](int v) { v %= N; return v < 0 ? v + N : v; };
        const Box b{ md(w.x0), md(w.y0), md(w.z0), w.nx, w.ny, w.nz };
        const size_t bytes = sizeof(double) * 10 * (size_t)w.nx * w.ny * w.nz;
        double *tmp = nullptr;
        cudaError_t e = cudaMallocAsync(&tmp, bytes, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return host_fail(e == cudaErrorMemoryAllocation ? AH_ERR_OOM : AH_ERR_CUDA, cudaGetErrorString(e));
        }
        e = launch_gather_window<float>(lat_fields(L), L.cur, N, b, tmp, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w.out, tmp, bytes, cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(tmp, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return host_fail(AH_ERR_CUDA, cudaGetErrorString(e));
        return AH_OK;
    }

    // Per-shape one-time set-up of the kernels this engine launches.
    cudaError_t prepare()
    {
        cudaError_t e = batch_shape_prepare(shape, num_sms, st, false);
        if (e == cudaSuccess && two) e = batch_shape_prepare(shape2, num_sms, st, true);
        return e;
    }

    // Observables of one lattice at its current step (the whole-lattice pass on
    // the step's tile walk; everything in FP64 if the near-cut list overflows);
    // they also choose the form of its next direct two-step launches.
    ah_status diag(Lat &L, ah_obs *out)
    {
        TraceRange tr("batch diagnostics");
        const View<float> v = lat_view(L);
        const Box b{ 0, 0, 0, L.N, L.N, L.N };
        const DiagCoef dc = host_diag_coef(L.cfg, L.step);
        if (fused_diag_ctas(L.N) > nparts) {
            char msg[160];
            snprintf(msg, sizeof msg, "diagnostics scratch too small: the N=%d pass needs %d partials, %d allocated",
                     L.N, fused_diag_ctas(L.N), nparts);
            return host_fail(AH_ERR_CUDA, msg);
        }
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
        L.weak = L.two && out->max_abs_theta <= kWeakTheta;
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

// Host copy of the device-side step counter, buffers and Pi/E set of an
// unfinished lattice after a round of R steps (R <= its steps to its next
// stop); returns the steps it advanced.
int advance_mirror(Lat &L, int R, bool two)
{
    if (!two || !L.two) {
        const int d = std::min(R, L.nsteps - L.step);
        L.step += d;
        L.cur ^= d & 1;
        return d;
    }
    // R / 2 two-step passes (each swaps the phi/theta buffers and the Pi/E set),
    // then, for an odd R, the single step if it leaves the lattice at its stop
    const int P = R / 2;
    const int single = (R % 2) && steps_to_event(L) - 2 * P == 1;
    L.step += 2 * P + single;
    L.cur ^= (P + single) & 1;
    L.pe ^= P & 1;
    return 2 * P + single;
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
extern "C" ah_status ah_batch_run_ex(const ah_config *cfgs, int32_t count, int32_t flags, ah_obs *series,
                                     int64_t series_cap, int64_t *series_len, ah_batch_stats *stats,
                                     const ah_window *windows, int32_t nwindows)
{
    if (!cfgs || count < 1 || (series && (series_cap < 1 || !series_len)) || nwindows < 0 || (nwindows && !windows))
        return host_fail(AH_ERR_ARG, "ah_batch_run: bad arguments");
    if (flags & ~(AH_BATCH_AUTOTUNE | AH_BATCH_NO_GRAPH | AH_BATCH_TWO_STEP))
        return host_fail(AH_ERR_ARG, "ah_batch_run: unknown flags");
    for (int i = 0; i < count; ++i) {
        ah_status st = check_batch_cfg(cfgs[i]);
        if (st != AH_OK) return st;
    }
    for (int k = 0; k < nwindows; ++k) {
        if (windows[k].lattice < 0 || windows[k].lattice >= count)
            return host_fail(AH_ERR_ARG, "window lattice index out of range");
        ah_status st = check_window(windows[k], cfgs[windows[k].lattice].N);
        if (st != AH_OK) return st;
    }
    const bool auto_pairs = (flags & AH_BATCH_TWO_STEP) != 0;
    bool two = false;
    for (int i = 0; i < count; ++i) two = two || lat_pairs(cfgs[i], auto_pairs);
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
    cudaError_t e = eng.init(!(flags & AH_BATCH_NO_GRAPH), two);
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        lats[i].cfg = cfgs[i];
        ptrs[i] = &lats[i];
        e = lat_setup(lats[i], lat_pairs(cfgs[i], auto_pairs), eng.st);
    }
    if (e != cudaSuccess) {
        cleanup();
        return host_fail(e == cudaErrorMemoryAllocation ? AH_ERR_OOM : AH_ERR_CUDA, cudaGetErrorString(e));
    }
    // shape: the fastest over two timed steps (two-step mode: two timed passes)
    // of the whole batch, states restored after
    int best = 0;
    if (flags & AH_BATCH_AUTOTUNE) {
        float best_ms = 0.0f;
        bool timed = false;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        const int nshapes = two ? batch2_shape_count() : batch_shape_count();
        for (int s = 0; s < nshapes && e == cudaSuccess; ++s) {
            bool ok = true;
            if (!two)
                for (auto &L : lats) ok = ok && batch_shape_ok(s, L.N);
            if (!ok) continue;
            (two ? eng.shape2 : eng.shape) = s;
            e = eng.prepare();
            if (e == cudaSuccess) e = eng.load(ptrs);
            if (e != cudaSuccess) break;
            eng.use_graph = false;
            const int R = two ? 4 : 2;
            e = eng.steps(R / 2);
            if (e == cudaSuccess) e = cudaEventRecord(a, eng.st);
            if (e == cudaSuccess) e = eng.steps(R);
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
        eng.weak_launches = 0;
        eng.rounds = 0;
    }
    (two ? eng.shape2 : eng.shape) = best;
    if (e == cudaSuccess) e = eng.prepare();
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
            advance_mirror(L, R, two);
            const bool due = L.step == L.nsteps || (L.cfg.diag_every > 0 && L.step % L.cfg.diag_every == 0);
            if (due) st = record(i);
        }
    }
    const double t2 = now_s();
    for (int k = 0; k < nwindows && st == AH_OK; ++k) st = eng.gather(lats[windows[k].lattice], windows[k]);
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->seconds = t2 - t1;
        stats->setup_seconds = t_setup;
        stats->site_updates = site_updates;
        stats->sims_per_hour = stats->seconds > 0 ? count * 3600.0 / stats->seconds : 0.0;
        stats->shape = best;
        stats->rounds = eng.rounds;
        stats->launches = eng.launches;
        stats->weak_field_launches = eng.weak_launches;
    }
    cleanup();
    return st;
}

extern "C" ah_status ah_batch_run(const ah_config *cfgs, int32_t count, int32_t flags, ah_obs *series,
                                  int64_t series_cap, int64_t *series_len, ah_batch_stats *stats)
{
    return ah_batch_run_ex(cfgs, count, flags, series, series_cap, series_len, stats, nullptr, 0);
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
    bool auto_pairs = false;  // AH_BATCH_TWO_STEP: pair the lattices with N >= kPairMinN

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
            const cudaError_t e = lat_setup(*L, lat_pairs(L->cfg, auto_pairs), eng.st);
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
        double su = 0.0;
        for (auto *L : loaded) su += (double)L->nsites * advance_mirror(*L, R, eng.two);
        {
            std::lock_guard<std::mutex> lk(mu);
            stats.site_updates += su;
            stats.launches = eng.launches;
        }
        // retire finished lattices with their final observables
        for (size_t i = 0; i < active.size();) {
            Lat &L = *active[i];
            if (L.step < L.nsteps) { ++i; continue; }
            ah_obs o;
            const ah_status ds = eng.diag(L, &o);
            std::lock_guard<std::mutex> lk(mu);
            Result &r = results[L.id];
            if (r.state != RQ_CANCELLED) {          // a cancel that arrived during its last round wins
                // the caller's window buffers are written under the lock, so a
                // cancel cannot return (and the caller free them) in between
                bool ok = ds == AH_OK || ds == AH_ERR_NONFINITE;
                for (const ah_window &w : L.wins)
                    if (ok) ok = eng.gather(L, w) == AH_OK;
                r.state = ok ? RQ_DONE : RQ_FAILED;
                if (!ok) r.err = "final diagnostics or a window read-back failed";
                r.obs = o;
                r.t_done = now_s() - t_origin;
            }
            cudaFreeAsync(L.mem, eng.st);
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
    if (!out || hbm_budget_bytes == 0 || max_slots < 1 || (flags & ~(AH_BATCH_NO_GRAPH | AH_BATCH_TWO_STEP)))
        return host_fail(AH_ERR_ARG, "ah_server_create: bad arguments");
    *out = nullptr;
    ah_server *s = new (std::nothrow) ah_server();
    if (!s) return host_fail(AH_ERR_OOM, "host allocation failed");
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->t_origin = now_s();
    if (const char *f = std::getenv("AH_FAKE_DEVICE_FAILURE_AFTER_ROUNDS")) s->fail_after_rounds = std::atoll(f);
    cudaGetDevice(&s->device);
    s->auto_pairs = (flags & AH_BATCH_TWO_STEP) != 0;
    // requests may ask for pairs themselves (AH_FLAG_TWO_STEP), so the engine
    // can always run two-step passes; without paired lattices it launches the
    // single-step kernel only, as in one-step mode
    cudaError_t e = s->eng.init(!(flags & AH_BATCH_NO_GRAPH), true);
    if (e == cudaSuccess) e = s->eng.prepare();
    if (e != cudaSuccess) {
        s->eng.release();
        delete s;
        return host_fail(AH_ERR_CUDA, cudaGetErrorString(e));
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return AH_OK;
}

ah_status ah_server_submit_ex(ah_server *s, const ah_config *cfg, const ah_window *windows, int32_t nwindows,
                              uint64_t *req_id)
{
    if (!s || !cfg || !req_id || nwindows < 0 || (nwindows && !windows))
        return host_fail(AH_ERR_ARG, "ah_server_submit: null argument");
    ah_status st = check_batch_cfg(*cfg);
    if (st != AH_OK) return st;
    for (int k = 0; k < nwindows; ++k)
        if ((st = check_window(windows[k], cfg->N)) != AH_OK) return st;
    auto L = std::make_unique<Lat>();
    L->cfg = *cfg;
    L->wins.assign(windows, windows + nwindows);
    L->bytes = lattice_bytes(*cfg, lat_pairs(*cfg, s->auto_pairs));
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

ah_status ah_server_submit(ah_server *s, const ah_config *cfg, uint64_t *req_id)
{
    return ah_server_submit_ex(s, cfg, nullptr, 0, req_id);
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
