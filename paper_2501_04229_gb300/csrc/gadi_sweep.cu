// gadi_sweep.cu -- batched GADI-IR: many (instance, alpha, omega) solves of
// constant-coefficient convection-diffusion systems in one persistent
// launch per size bin, captured in a CUDA graph.
//
// Teams of k blocks take work items from a global queue (largest systems
// first, each instance's candidates from the middle of its list outwards)
// and run one complete FP16-inner GADI-IR solve per item: a team of one
// block uses block-level reductions only; a team of k > 1 blocks shares
// its rows over its blocks and synchronises through a team-scoped exchange
// (the grid exchange of the solve kernel, on the team's own counter and
// partials). The system of an item is built on the device from (dim, N,
// beta): the operator is the matrix-free stencil, b = A 1 (the paper's
// right-hand side), x0 = 0. With racing on, a solve stops once it has used
// more operator applications than a finished candidate of the same instance
// (the record says so): such a candidate cannot be the best one.
//
// Schedule (row bins and tiles): instances are binned by their number of
// rows; each bin runs as its own launch with one team size k and one block
// size. Both come from a small autotuner: for each bin it times short probes
// of the bin's largest items (outer steps capped) over the bin's team sizes
// and block sizes 128 / 256 / 512, and keeps the fastest, cached per (dim,
// items-per-row, bin, largest n).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/gadi.h"
#include "gadi_solve.cuh"

using namespace gadi;

namespace {

struct SweepItem {
    int inst, cand;
};

struct SweepArgs {
    const gadi_sweep_instance *inst;
    const gadi_sweep_candidate *cand;
    const SweepItem *items;
    int nitems;
    int *next;                     // [0] the queue head, [1] the first error (a wait that expired)
    long long *best;
    gadi_sweep_record *rec;
    unsigned char *scratch;        // per team: Ctl, partials, vectors
    size_t per_team, part_off, vec_off;
    int team;                      // blocks per team
    int64_t maxn;
    double tol, eps;
    int max_inner, max_outer, race;
    unsigned long long wait_ns;
};

__host__ __device__ inline int half_scale_hd(double norm, double sigma)
{
    double v = norm + fabs(sigma);
    if (!(v > 0.0) || !isfinite(v)) return 0;
    int e;
    double m = frexp(v, &e);
    return ((m == 0.5) ? e - 1 : e) - 1;
}

// max over rows of the summed |coefficients| (ascending column order), by row class
__host__ __device__ inline double row_norm_hd(int dim, int N, double lo, double dg, double hi)
{
    double best = 0.0;
    int classes = dim == 3 ? 27 : 9;
    for (int cls = 0; cls < classes; ++cls) {
        int pos[3] = {0, 0, 0}, t = cls;
        bool ok = true;
        for (int d = 0; d < dim; ++d) {
            pos[d] = t % 3;
            t /= 3;
            if (pos[d] == 1 && N < 3) ok = false;
            if (pos[d] == 2 && N < 2) ok = false;
        }
        if (!ok) continue;
        double s = 0.0;
        for (int d = dim - 1; d >= 0; --d)
            if (pos[d] != 0) s += fabs(lo);
        s += fabs(dg);
        for (int d = 0; d < dim; ++d)
            if (pos[d] != 2 && N >= 2) s += fabs(hi);
        best = fmax(best, s);
    }
    return best;
}

struct XOnes64 {
    __device__ __forceinline__ double one(int64_t) const { return 1.0; }
    template <int K>
    __device__ __forceinline__ void many(int64_t, double (&o)[K]) const
    {
#pragma unroll
        for (int k = 0; k < K; ++k) o[k] = 1.0;
    }
};

template <int DIM, int R>
__global__ void __launch_bounds__(512, 1) gadi_sweep_kernel(const SweepArgs s)
{
    using Op = StencilOp<__half, DIM, R>;
    const unsigned k = (unsigned)s.team;
    const unsigned team = blockIdx.x / k, rank = blockIdx.x % k;
    unsigned char *mine = s.scratch + (size_t)team * s.per_team;
    Ctl *ctl = reinterpret_cast<Ctl *>(mine);
    double *part = reinterpret_cast<double *>(mine + s.part_off);
    double *bvec = reinterpret_cast<double *>(mine + s.vec_off);
    double *xvec = bvec + s.maxn;
    double *r64 = xvec + s.maxn;
    double *x2 = r64 + s.maxn;
    float *r32 = reinterpret_cast<float *>(x2 + s.maxn);
    __half *V = reinterpret_cast<__half *>(r32 + s.maxn);
    GridExchange ex{ctl, part, 0u, s.wait_ns, 0u, k == 1};
    ex.team = k;
    ex.rank = rank;
    const int64_t t0 = (int64_t)rank * blockDim.x + threadIdx.x, nt = (int64_t)k * blockDim.x;
    const bool lead = rank == 0 && threadIdx.x == 0;
    // a wait that expired leaves the team's exchange out of step: the team
    // records the error and stops
    auto fail = [&]() {
        if (lead) atomicCAS(s.next + 1, 0, kErrTimeout);
    };
    for (;;) {
        // the team's next item: its first block takes it from the queue and
        // the exchange (a maximum) hands it to the other blocks
        double iv[1] = {-1.0};
        if (lead) iv[0] = (double)atomicAdd(s.next, 1);
        {
            const int opsI[1] = {kMax};
            if (!ex.allreduce(iv, opsI)) { fail(); return; }
        }
        const int item = (int)iv[0];
        if (item >= s.nitems) return;
        const SweepItem wi = s.items[item];
        const gadi_sweep_instance in = s.inst[wi.inst];
        const gadi_sweep_candidate cd = s.cand[wi.cand];
        const int N = in.N;
        const int64_t n = DIM == 3 ? (int64_t)N * N * N : (int64_t)N * N;
        // the operator as the HSS split of the assembled matrix gives it
        const double c = in.beta * (1.0 / (N + 1)) / 2.0;
        const double a_diag = 2.0 * DIM, a_lo = -1.0 - c, a_hi = -1.0 + c;
        const double m_off = 0.5 * (a_hi + a_lo), n_up = 0.5 * (a_hi - a_lo);
        const int sM = half_scale_hd(row_norm_hd(DIM, N, m_off, a_diag, m_off), cd.alpha);
        const int sN = half_scale_hd(row_norm_hd(DIM, N, -n_up, 0.0, n_up), cd.alpha);
        const double scM = ldexp(1.0, -sM), scN = ldexp(1.0, -sN);
        Op op{};
        op.dim = DIM;
        op.N = N;
        op.divN = div_magic((unsigned)op.N);
        op.n = n;
        op.a_diag = a_diag;
        op.a_lo = a_lo;
        op.a_hi = a_hi;
        op.h_diag = __half2float(__double2half(a_diag * scM));
        op.h_off = __half2float(__double2half(m_off * scM));
        op.s_c = __half2float(__double2half(n_up * scN));
        op.sigH = (float)ldexp(cd.alpha, -sM);
        op.sigS = (float)ldexp(cd.alpha, -sN);
        const int64_t nitems = n / R;

        // b = A 1, x0 = 0, ||b||_inf
        double bm[1] = {0.0};
        {
            const XOnes64 ones;
            for (int64_t it = t0; it < nitems; it += nt) {
                double o[R], z[R];
                op.rowsA(it, ones, o);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    bm[0] = fmax(bm[0], fabs(o[q]));
                    z[q] = 0.0;
                }
                ItemIO64<R>::st(bvec, it, o);
                ItemIO64<R>::st(xvec, it, z);
            }
            const int opsm[1] = {kMax};
            if (!ex.allreduce(bm, opsm)) { fail(); return; }
        }
        if (lead) ctl->status = kErrNotConverged;

        SolveArgs<Op, __half> a;
        a.op = op;
        a.n = n;
        a.nitems = nitems;
        a.b = bvec;
        a.x = xvec;
        a.x2 = x2;
        a.r64 = r64;
        a.r32 = r32;
        for (int j = 0; j < 9; ++j) a.v[j] = V + j * s.maxn;
        a.anorm = row_norm_hd(DIM, N, a_lo, a_diag, a_hi);
        a.bnorm = bm[0];
        a.tol = s.tol;
        a.eps = s.eps;
        a.pfac = (2.0 - cd.omega) * cd.alpha;
        a.sM = sM;
        a.sN = sN;
        a.half = 1;
        a.naive = 0;
        a.stop_kind = 0;
        a.max_inner = s.max_inner;
        a.max_outer = s.max_outer;
        a.ctl = ctl;
        a.part = part;
        a.eta_hist = nullptr;
        a.race_bound = s.race ? s.best + wi.inst : nullptr;
        a.wait_ns = s.wait_ns;
        a.extra = 0;
        a.zlen = 0;
        const unsigned long long t_start = global_ns();
        solve_body(a, ex, t0, nt, lead);
        __syncthreads();
        if (ld_volatile_i32(&ctl->error) != 0) { fail(); return; }
        if (lead) {
            gadi_sweep_record r;
            r.instance = wi.inst;
            r.candidate = wi.cand;
            r.raced_out = ctl->status == kRacedOut;
            r.status = r.raced_out ? kErrNotConverged : ctl->status;
            r.outer_iters = ctl->outer_iters;
            r.team_blocks = (int)k;
            r.inner_iters_H = ctl->itH;
            r.inner_iters_S = ctl->itS;
            r.spmv_count = ctl->spmv;
            r.eta_inf = ctl->eta;
            r.time_ms = (double)(global_ns() - t_start) * 1e-6;
            s.rec[item] = r;
            if (r.status == kOk) atomicMin(s.best + wi.inst, (long long)ctl->spmv);
        }
    }
}

template <int DIM, int R>
const void *sweep_kernel_ptr()
{
    return (const void *)gadi_sweep_kernel<DIM, R>;
}

const void *pick_kernel(int dim, int r)
{
    if (dim == 3) return r == 8 ? sweep_kernel_ptr<3, 8>() : sweep_kernel_ptr<3, 1>();
    return r == 8 ? sweep_kernel_ptr<2, 8>() : sweep_kernel_ptr<2, 1>();
}

std::mutex g_tune_mu;
// (dim, R, bin, max n, fixed block threads, fixed team blocks) -> (block threads, team blocks)
std::map<std::tuple<int, int, int, int64_t, int, int>, std::pair<int, int>> g_tuned;

// row bins of the schedule and the team sizes tried in each
constexpr int kBins = 4;
int bin_of(int64_t n)
{
    return n < (1 << 15) ? 0 : (n < (1 << 18) ? 1 : (n < (1 << 20) ? 2 : 3));
}
const std::vector<int> &bin_teams(int bin)
{
    static const std::vector<int> t[kBins] = {{1}, {1, 2, 4}, {2, 4, 8}, {4, 8, 16}};
    return t[bin];
}

struct Group {
    int dim, r, bin;
    std::vector<SweepItem> items;
    int64_t maxn;
};

struct DevBuf {
    void *p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

#define SW_CK(call)                                                                           \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            cudaGetLastError();                                                               \
            return e_ == cudaErrorMemoryAllocation ? GADI_ERR_OUT_OF_MEMORY : GADI_ERR_CUDA;  \
        }                                                                                     \
    } while (0)

// blocks that fit at once for a block size
int resident_blocks(const void *kern, int threads)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0);
    return per * sms;
}

// run the items of one group with teams of `team` blocks: a graph with the
// reset of the queue, the error flag and every team's control block, then
// the cooperative launch (all blocks co-resident, as the team exchanges
// need)
gadi_status run_group(const Group &g, int threads, int team, const gadi_sweep_instance *dinst,
                      const gadi_sweep_candidate *dcand, long long *dbest, double tol, double eps,
                      int max_inner, int max_outer, int race, cudaStream_t stream,
                      gadi_sweep_record *hrec_out)
{
    const void *kern = pick_kernel(g.dim, g.r);
    const int nitems = (int)g.items.size();
    const int resident = resident_blocks(kern, threads);
    if (team < 1 || resident < team) return GADI_ERR_INVALID_ARG;
    const int teams = std::min(resident / team, nitems);
    const int blocks = teams * team;
    const size_t part_off = 256;
    const size_t vec_off = part_off + ((size_t)2 * kMaxSlots * team * sizeof(double) + 255) / 256 * 256;
    const size_t per_team =
        (vec_off + (size_t)g.maxn * (4 * sizeof(double) + sizeof(float) + 9 * sizeof(__half)) + 255) / 256 * 256;
    DevBuf items, next, rec, scratch;
    SW_CK(cudaMalloc(&items.p, nitems * sizeof(SweepItem)));
    SW_CK(cudaMalloc(&next.p, 2 * sizeof(int)));
    SW_CK(cudaMalloc(&rec.p, nitems * sizeof(gadi_sweep_record)));
    SW_CK(cudaMalloc(&scratch.p, per_team * teams));
    SW_CK(cudaMemcpyAsync(items.p, g.items.data(), nitems * sizeof(SweepItem), cudaMemcpyHostToDevice, stream));
    SweepArgs a;
    a.inst = dinst;
    a.cand = dcand;
    a.items = (const SweepItem *)items.p;
    a.nitems = nitems;
    a.next = (int *)next.p;
    a.best = dbest;
    a.rec = (gadi_sweep_record *)rec.p;
    a.scratch = (unsigned char *)scratch.p;
    a.per_team = per_team;
    a.part_off = part_off;
    a.vec_off = vec_off;
    a.team = team;
    a.maxn = g.maxn;
    a.tol = tol;
    a.eps = eps;
    a.max_inner = max_inner;
    a.max_outer = max_outer;
    a.race = race;
    a.wait_ns = 2000000000ULL;
    // capture the resets and the launch in a graph, on a stream of our own
    cudaStream_t cap;
    SW_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *args[] = {(void *)&a};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = cap;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(next.p, 0, 2 * sizeof(int), cap);
        cudaMemset2DAsync(scratch.p, per_team, 0, sizeof(Ctl), teams, cap);
        cudaLaunchKernelExC(&cfg, kern, args);
        e = cudaStreamEndCapture(cap, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);     // inputs uploaded on the caller's stream
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, stream);
    int flags[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hrec_out, rec.p, nitems * sizeof(gadi_sweep_record),
                                              cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags, next.p, sizeof flags, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GADI_ERR_CUDA;
    }
    if (flags[1] != 0) return GADI_ERR_TIMEOUT;
    return GADI_OK;
}

}  // namespace

extern "C" gadi_status gadi_sweep(const gadi_sweep_instance *inst, int32_t ninst,
                                  const gadi_sweep_candidate *cand, int32_t ncand, double tol,
                                  double eps_inner, int32_t max_inner, int32_t max_outer, int32_t race,
                                  int32_t block_threads, int32_t team_blocks, void *cuda_stream,
                                  gadi_sweep_record *records)
{
    if (!inst || !cand || !records || ninst < 1 || ncand < 1) return GADI_ERR_INVALID_ARG;
    if ((int64_t)ninst * ncand > (1 << 26)) return GADI_ERR_INVALID_ARG;
    if (!(tol > 0.0) || !(eps_inner > 0.0 && eps_inner < 1.0) || max_inner < 1 || max_outer < 0)
        return GADI_ERR_INVALID_ARG;
    if (block_threads != 0 && block_threads != 128 && block_threads != 256 && block_threads != 512)
        return GADI_ERR_INVALID_ARG;
    if (team_blocks < 0 || team_blocks > 64) return GADI_ERR_INVALID_ARG;
    for (int i = 0; i < ninst; ++i) {
        const gadi_sweep_instance &s = inst[i];
        if ((s.dim != 2 && s.dim != 3) || s.N < 1 || !std::isfinite(s.beta)) return GADI_ERR_INVALID_ARG;
        const int64_t n = s.dim == 3 ? (int64_t)s.N * s.N * s.N : (int64_t)s.N * s.N;
        if (n >= (1LL << 31)) return GADI_ERR_INVALID_ARG;
    }
    for (int j = 0; j < ncand; ++j)
        if (!(cand[j].alpha > 0.0) || !std::isfinite(cand[j].alpha) || !(cand[j].omega >= 0.0 && cand[j].omega < 2.0))
            return GADI_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // groups by (dim, items of 8 rows or 1, row bin), items largest first
    std::vector<Group> groups;
    auto nrows = [&](int i) { return inst[i].dim == 3 ? (int64_t)inst[i].N * inst[i].N * inst[i].N
                                                       : (int64_t)inst[i].N * inst[i].N; };
    for (int i = 0; i < ninst; ++i) {
        const int r = inst[i].N % 8 == 0 ? 8 : 1;
        const int bin = bin_of(nrows(i));
        auto it = std::find_if(groups.begin(), groups.end(), [&](const Group &g) {
            return g.dim == inst[i].dim && g.r == r && g.bin == bin;
        });
        if (it == groups.end()) {
            groups.push_back(Group{inst[i].dim, r, bin, {}, 0});
            it = groups.end() - 1;
        }
        for (int j = 0; j < ncand; ++j) it->items.push_back(SweepItem{i, j});
        it->maxn = std::max(it->maxn, nrows(i));
    }
    for (auto &g : groups)
        // largest systems first; within an instance the candidates from the
        // middle of the list outwards (the list is ordered by alpha, and the
        // middle is where optima usually lie), so that a cheap finished
        // candidate sets the race bound early
        std::stable_sort(g.items.begin(), g.items.end(), [&](const SweepItem &a, const SweepItem &b) {
            if (nrows(a.inst) != nrows(b.inst)) return nrows(a.inst) > nrows(b.inst);
            if (a.inst != b.inst) return a.inst < b.inst;
            return std::abs(2 * a.cand - (ncand - 1)) < std::abs(2 * b.cand - (ncand - 1));
        });

    DevBuf dinst, dcand, dbest;
    SW_CK(cudaMalloc(&dinst.p, ninst * sizeof(gadi_sweep_instance)));
    SW_CK(cudaMalloc(&dcand.p, ncand * sizeof(gadi_sweep_candidate)));
    SW_CK(cudaMalloc(&dbest.p, ninst * sizeof(long long)));
    SW_CK(cudaMemcpyAsync(dinst.p, inst, ninst * sizeof(gadi_sweep_instance), cudaMemcpyHostToDevice, stream));
    SW_CK(cudaMemcpyAsync(dcand.p, cand, ncand * sizeof(gadi_sweep_candidate), cudaMemcpyHostToDevice, stream));
    std::vector<long long> hbest(ninst, LLONG_MAX);
    SW_CK(cudaMemcpyAsync(dbest.p, hbest.data(), ninst * sizeof(long long), cudaMemcpyHostToDevice, stream));

    for (auto &g : groups) {
        int threads = block_threads, team = team_blocks;
        if (threads == 0 || team == 0) {
            const auto key = std::make_tuple(g.dim, g.r, g.bin, g.maxn, block_threads, team_blocks);
            std::pair<int, int> pick{0, 0};
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto f = g_tuned.find(key);
                if (f != g_tuned.end()) pick = f->second;
            }
            if (pick.first == 0) {
                // probe: the bin's largest items (enough to fill the teams of
                // the smallest team size), outer steps capped, racing off
                const std::vector<int> tcand = block_threads ? std::vector<int>{block_threads}
                                                             : std::vector<int>{128, 256, 512};
                const std::vector<int> kcand = team_blocks ? std::vector<int>{team_blocks} : bin_teams(g.bin);
                Group probe{g.dim, g.r, g.bin, {}, g.maxn};
                const int np = std::min<int>((int)g.items.size(), 2 * resident_blocks(pick_kernel(g.dim, g.r), 512) /
                                                                      std::max(1, kcand.front()));
                probe.items.assign(g.items.begin(), g.items.begin() + std::max(1, np));
                std::vector<gadi_sweep_record> tmp(probe.items.size());
                double best_t = 1e300;
                for (int tt : tcand)
                    for (int kk : kcand) {
                        if (resident_blocks(pick_kernel(g.dim, g.r), tt) < kk) continue;
                        const auto t0 = std::chrono::steady_clock::now();
                        gadi_status st = run_group(probe, tt, kk, (gadi_sweep_instance *)dinst.p,
                                                   (gadi_sweep_candidate *)dcand.p, (long long *)dbest.p, tol,
                                                   eps_inner, max_inner, std::min(max_outer, 8), 0, stream,
                                                   tmp.data());
                        if (st != GADI_OK) return st;
                        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                        if (dt < best_t) {
                            best_t = dt;
                            pick = {tt, kk};
                        }
                    }
                if (pick.first == 0) return GADI_ERR_INVALID_ARG;   // no team size fits
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tuned[key] = pick;
            }
            threads = block_threads ? block_threads : pick.first;
            team = team_blocks ? team_blocks : pick.second;
        }
        std::vector<gadi_sweep_record> recs(g.items.size());
        gadi_status st = run_group(g, threads, team, (gadi_sweep_instance *)dinst.p, (gadi_sweep_candidate *)dcand.p,
                                   (long long *)dbest.p, tol, eps_inner, max_inner, max_outer, race, stream,
                                   recs.data());
        if (st != GADI_OK) return st;
        for (const auto &r : recs) records[(size_t)r.instance * ncand + r.candidate] = r;
    }
    return GADI_OK;
}
