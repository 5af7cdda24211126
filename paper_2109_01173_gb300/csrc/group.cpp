// Heterogeneous batches: problems of any (k, n, bc), grouped into batched handles
// of equal (k, n, bc) (each group one batched MO-PCG: shared t-factors and Q2,
// per-instance s-factors, Q1, lambda, gamma, profiles), solved concurrently on
// one stream per group from host threads.  The number of groups in flight is a
// run-time choice: mofem_group_autotune times the candidates on a real solve and
// keeps the fastest.
#include "internal.h"

#include <algorithm>
#include <chrono>
#include <map>
#include <atomic>
#include <thread>
#include <tuple>
#include <vector>

struct mofem_group_ctx {
    struct Group {
        int k = 0, n = 0, q = 0;
        mofem_bc bc = MOFEM_BC_DIRICHLET;
        std::vector<int> members;     // problem indices, in input order
        mofem_handle h = nullptr;
        cudaStream_t st = nullptr;
        double* F = nullptr;          // [B][n][n]
        double* U = nullptr;          // [B][q][q]
    };
    int count = 0;
    int concurrency = -1;             // -1: all groups in lockstep (one graph, one GEMM launch per
                                      // iteration); else groups solved apart, this many at once (0: all)
    int apply_tile_div = 1;           // operator-apply tile height of every group: one wave of CTAs / this
    std::vector<Group> groups;
    FusedState fused;                 // lockstep graph and descriptors, kept between solves
    cudaStream_t st = nullptr;        // the lockstep solve's stream
};

namespace {

// Group key: (k, n, bc); groups ordered by decreasing work (n^3 * size) so the
// largest start first.
void make_layout(int count, const mofem_problem* p, std::vector<std::vector<int>>& out) {
    std::map<std::tuple<int, int, int>, std::vector<int>> m;
    for (int i = 0; i < count; ++i) m[std::make_tuple(p[i].k, p[i].n_nodes, (int)p[i].bc)].push_back(i);
    out.clear();
    for (auto& kv : m) out.push_back(kv.second);
    std::stable_sort(out.begin(), out.end(), [&](const std::vector<int>& a, const std::vector<int>& b) {
        const double wa = (double)p[a[0]].n_nodes * p[a[0]].n_nodes * p[a[0]].n_nodes * a.size();
        const double wb = (double)p[b[0]].n_nodes * p[b[0]].n_nodes * p[b[0]].n_nodes * b.size();
        return wa > wb;
    });
}

void free_group(mofem_group_ctx* g) {
    fused_free(&g->fused);
    if (g->st) cudaStreamDestroy(g->st);
    for (auto& gr : g->groups) {
        if (gr.h) mofem_destroy(gr.h);
        cudaFree(gr.F);
        cudaFree(gr.U);
        if (gr.st) cudaStreamDestroy(gr.st);
    }
    delete g;
}

}  // namespace

extern "C" mofem_status mofem_group_layout(int count, const mofem_problem* problems, int* n_groups, int* group_of) {
    if (count < 1 || !problems || !n_groups) return MOFEM_ERR_INVALID_ARG;
    std::vector<std::vector<int>> lay;
    make_layout(count, problems, lay);
    *n_groups = (int)lay.size();
    if (group_of)
        for (size_t gi = 0; gi < lay.size(); ++gi)
            for (int i : lay[gi]) group_of[i] = (int)gi;
    return MOFEM_OK;
}

extern "C" mofem_status mofem_group_setup(int count, const mofem_problem* problems, const mofem_opts* opts,
                                          mofem_group* out) {
    if (count < 1 || !problems || !out) return MOFEM_ERR_INVALID_ARG;
    *out = nullptr;
    auto* g = new (std::nothrow) mofem_group_ctx();
    if (!g) return MOFEM_ERR_OOM;
    g->count = count;
    std::vector<std::vector<int>> lay;
    make_layout(count, problems, lay);
    for (auto& mem : lay) {
        mofem_group_ctx::Group gr;
        const mofem_problem& p0 = problems[mem[0]];
        gr.k = p0.k;
        gr.n = p0.n_nodes;
        gr.bc = p0.bc;
        gr.members = mem;
        std::vector<mofem_profile> g1, g2;
        std::vector<double> gam;
        for (int i : mem) {
            g1.push_back(problems[i].g1);
            g2.push_back(problems[i].g2);
            gam.push_back(problems[i].gamma);
        }
        mofem_status s = cudaStreamCreateWithFlags(&gr.st, cudaStreamNonBlocking) == cudaSuccess ? MOFEM_OK
                                                                                                : MOFEM_ERR_CUDA;
        if (s == MOFEM_OK)
            s = mofem_setup_batched((int)mem.size(), g1.data(), g2.data(), gr.k, gr.n, gam.data(), gr.bc, opts, gr.st,
                                    &gr.h);
        if (s == MOFEM_OK) {
            gr.q = gr.h->q;
            s = solver_init(gr.h, gr.st);   // scratch that later calls only look up (threads)
        }
        const size_t B = mem.size();
        if (s == MOFEM_OK && cudaMalloc(&gr.F, sizeof(double) * B * gr.n * gr.n) != cudaSuccess) s = MOFEM_ERR_OOM;
        if (s == MOFEM_OK && cudaMalloc(&gr.U, sizeof(double) * B * gr.q * gr.q) != cudaSuccess) s = MOFEM_ERR_OOM;
        g->groups.push_back(gr);
        if (s != MOFEM_OK) {
            free_group(g);
            return s;
        }
    }
    *out = g;
    return MOFEM_OK;
}

// All groups in lockstep on one stream (solve_fused): MOFEM_ERR_UNSUPPORTED when that form
// does not apply (FP64, or an FP16 inner solve that needs the TF32 retry), the caller's U
// untouched then.
static mofem_status solve_lockstep(mofem_group g, const double* const* F, double* const* U, double rtol, int max_iter,
                                   mofem_precision prec, mofem_solve_info* infos, cudaStream_t stream) {
    if (prec == MOFEM_FP64) return MOFEM_ERR_UNSUPPORTED;
    if (!g->st) MOFEM_CUDA_TRY(cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking));
    cudaEvent_t ev_in = nullptr;
    MOFEM_CUDA_TRY(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
    MOFEM_CUDA_TRY(cudaEventRecord(ev_in, stream));
    MOFEM_CUDA_TRY(cudaStreamWaitEvent(g->st, ev_in, 0));
    cudaEventDestroy(ev_in);
    const int ng = (int)g->groups.size();
    std::vector<mofem_ctx*> cs(ng);
    std::vector<const double*> Fg(ng);
    std::vector<double*> Ug(ng);
    for (int gi = 0; gi < ng; ++gi) {
        auto& gr = g->groups[gi];
        const size_t nn = (size_t)gr.n * gr.n, qq = (size_t)gr.q * gr.q;
        for (size_t j = 0; j < gr.members.size(); ++j) {
            const int i = gr.members[j];
            MOFEM_CUDA_TRY(cudaMemcpyAsync(gr.F + j * nn, F[i], sizeof(double) * nn, cudaMemcpyDeviceToDevice, g->st));
            MOFEM_CUDA_TRY(cudaMemcpyAsync(gr.U + j * qq, U[i], sizeof(double) * qq, cudaMemcpyDeviceToDevice, g->st));
        }
        cs[gi] = gr.h;
        Fg[gi] = gr.F;
        Ug[gi] = gr.U;
    }
    std::vector<mofem_solve_info> gi_info(ng);
    const mofem_status s = solve_fused(cs.data(), ng, Fg.data(), Ug.data(), rtol, max_iter, prec, &g->fused,
                                       gi_info.data(), g->st);
    if (s != MOFEM_OK && s != MOFEM_ERR_NOT_CONVERGED) return s;
    for (int gi = 0; gi < ng; ++gi) {
        auto& gr = g->groups[gi];
        const size_t qq = (size_t)gr.q * gr.q;
        for (size_t j = 0; j < gr.members.size(); ++j)
            MOFEM_CUDA_TRY(cudaMemcpyAsync(U[gr.members[j]], gr.U + j * qq, sizeof(double) * qq,
                                           cudaMemcpyDeviceToDevice, g->st));
        if (infos)
            for (int i : gr.members) infos[i] = gi_info[gi];
    }
    MOFEM_CUDA_TRY(cudaStreamSynchronize(g->st));
    return s;
}

extern "C" mofem_status mofem_group_solve(mofem_group g, const double* const* F, double* const* U, double rtol,
                                          int max_iter, mofem_precision prec, mofem_solve_info* infos,
                                          cudaStream_t stream) {
    if (!g || !F || !U || !(rtol > 0.0) || max_iter < 1) return MOFEM_ERR_INVALID_ARG;
    for (int i = 0; i < g->count; ++i)
        if (!F[i] || !U[i]) return MOFEM_ERR_INVALID_ARG;
    if (g->concurrency < 0) {
        const mofem_status s = solve_lockstep(g, F, U, rtol, max_iter, prec, infos, stream);
        if (s != MOFEM_ERR_UNSUPPORTED) return s;
        // otherwise: the groups apart, all at once
    }
    // groups start after the caller's prior work on `stream`
    cudaEvent_t ev_in = nullptr;
    if (cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming) != cudaSuccess) return MOFEM_ERR_CUDA;
    if (cudaEventRecord(ev_in, stream) != cudaSuccess) {
        cudaEventDestroy(ev_in);
        return MOFEM_ERR_CUDA;
    }
    const int ng = (int)g->groups.size();
    std::vector<mofem_status> res(ng, MOFEM_OK);
    int dev = 0;
    cudaGetDevice(&dev);
    auto run = [&](int gi) {
        cudaSetDevice(dev);
        auto& gr = g->groups[gi];
        mofem_status s = cudaStreamWaitEvent(gr.st, ev_in, 0) == cudaSuccess ? MOFEM_OK : MOFEM_ERR_CUDA;
        const size_t nn = (size_t)gr.n * gr.n, qq = (size_t)gr.q * gr.q;
        for (size_t j = 0; j < gr.members.size() && s == MOFEM_OK; ++j) {
            const int i = gr.members[j];
            if (cudaMemcpyAsync(gr.F + j * nn, F[i], sizeof(double) * nn, cudaMemcpyDeviceToDevice, gr.st) !=
                    cudaSuccess ||
                cudaMemcpyAsync(gr.U + j * qq, U[i], sizeof(double) * qq, cudaMemcpyDeviceToDevice, gr.st) !=
                    cudaSuccess)
                s = MOFEM_ERR_CUDA;
        }
        mofem_solve_info info{};
        if (s == MOFEM_OK) s = solve_elliptic(gr.h, gr.F, gr.U, rtol, max_iter, prec, &info, gr.st);
        const mofem_status solve_s = s;
        if (s == MOFEM_OK || s == MOFEM_ERR_NOT_CONVERGED) {
            for (size_t j = 0; j < gr.members.size(); ++j)
                if (cudaMemcpyAsync(U[gr.members[j]], gr.U + j * qq, sizeof(double) * qq, cudaMemcpyDeviceToDevice,
                                    gr.st) != cudaSuccess)
                    s = MOFEM_ERR_CUDA;
            if (cudaStreamSynchronize(gr.st) != cudaSuccess) s = MOFEM_ERR_CUDA;
            if (s == MOFEM_OK) s = solve_s;
        }
        if (infos)
            for (int i : gr.members) {
                infos[i] = info;
                infos[i].status = s;
            }
        res[gi] = s;
    };
    // `width` workers take the next group (largest first) as soon as they are free
    const int width = g->concurrency > 0 ? std::min(g->concurrency, ng) : ng;
    if (g->concurrency < 0) cudaStreamSynchronize(g->st);   // a lockstep attempt's copies are done
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    for (int w = 0; w < width; ++w)
        th.emplace_back([&]() {
            for (int gi = next.fetch_add(1); gi < ng; gi = next.fetch_add(1)) run(gi);
        });
    for (auto& t : th) t.join();
    cudaEventDestroy(ev_in);
    mofem_status worst = MOFEM_OK;
    for (auto s : res)
        if (s != MOFEM_OK && (worst == MOFEM_OK || worst == MOFEM_ERR_NOT_CONVERGED)) worst = s;
    return worst;
}

extern "C" mofem_status mofem_group_autotune(mofem_group g, const double* const* F, double* const* U, double rtol,
                                             int max_iter, mofem_precision prec, int* chosen) {
    if (!g) return MOFEM_ERR_INVALID_ARG;
    const int ng = (int)g->groups.size();
    // candidates (mode, apply tile divisor): lockstep with one-wave or half-height apply tiles
    // (the mixed forms), then the groups apart, 1 .. all in flight
    std::vector<std::pair<int, int>> cand;
    if (prec != MOFEM_FP64) {
        cand.push_back({-1, 1});
        cand.push_back({-1, 2});
    }
    for (int c : {1, 2, 4, 8, 16})
        if (c < ng) cand.push_back({c, 1});
    cand.push_back({ng, 1});
    auto set_tile = [&](int div) {
        if (div == g->apply_tile_div) return;
        g->apply_tile_div = div;
        for (auto& gr : g->groups) set_apply_seg_div(gr.h, div);
        if (g->fused.loop) {   // the lockstep graph holds the old apply grids
            cudaGraphExecDestroy(g->fused.loop);
            g->fused.loop = nullptr;
        }
    };
    // every candidate starts from the caller's initial guesses (saved here)
    std::vector<size_t> off(g->count + 1, 0);
    for (auto& gr : g->groups)
        for (int i : gr.members) off[i + 1] = (size_t)gr.q * gr.q;
    for (int i = 0; i < g->count; ++i) off[i + 1] += off[i];
    double* save = nullptr;
    if (cudaMalloc(&save, sizeof(double) * off[g->count]) != cudaSuccess) return MOFEM_ERR_OOM;
    auto copy_all = [&](bool to_save) {
        for (int i = 0; i < g->count; ++i) {
            const size_t bytes = sizeof(double) * (off[i + 1] - off[i]);
            if (to_save) cudaMemcpy(save + off[i], U[i], bytes, cudaMemcpyDeviceToDevice);
            else cudaMemcpy(U[i], save + off[i], bytes, cudaMemcpyDeviceToDevice);
        }
    };
    copy_all(true);
    g->concurrency = ng;   // warm-up: operand copies, graphs and scratch of every group
    mofem_status s = mofem_group_solve(g, F, U, rtol, max_iter, prec, nullptr, nullptr);
    if ((s == MOFEM_OK || s == MOFEM_ERR_NOT_CONVERGED) && prec != MOFEM_FP64) {   // and of the lockstep form
        copy_all(false);
        g->concurrency = -1;
        s = mofem_group_solve(g, F, U, rtol, max_iter, prec, nullptr, nullptr);
    }
    double best = 1e300;
    std::pair<int, int> best_c{ng, 1};
    for (size_t ci = 0; ci < cand.size() && (s == MOFEM_OK || s == MOFEM_ERR_NOT_CONVERGED); ++ci) {
        copy_all(false);
        g->concurrency = cand[ci].first;
        set_tile(cand[ci].second);
        if (cand[ci].second != 1) {   // a new tile height: one untimed solve builds its graphs
            s = mofem_group_solve(g, F, U, rtol, max_iter, prec, nullptr, nullptr);
            copy_all(false);
            if (s != MOFEM_OK && s != MOFEM_ERR_NOT_CONVERGED) break;
        }
        const auto t0 = std::chrono::steady_clock::now();
        s = mofem_group_solve(g, F, U, rtol, max_iter, prec, nullptr, nullptr);
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dt < best) {
            best = dt;
            best_c = cand[ci];
        }
    }
    copy_all(false);
    cudaFree(save);
    g->concurrency = best_c.first;
    set_tile(best_c.second);
    if (chosen) *chosen = best_c.first;
    return (s == MOFEM_OK || s == MOFEM_ERR_NOT_CONVERGED) ? MOFEM_OK : s;
}

extern "C" mofem_status mofem_group_set_mode(mofem_group g, int mode) {
    if (!g || mode < -1) return MOFEM_ERR_INVALID_ARG;
    g->concurrency = mode;
    return MOFEM_OK;
}

extern "C" mofem_status mofem_group_get_tuning(mofem_group g, int* mode, int* apply_tile_div) {
    if (!g) return MOFEM_ERR_INVALID_ARG;
    if (mode) *mode = g->concurrency;
    if (apply_tile_div) *apply_tile_div = g->apply_tile_div;
    return MOFEM_OK;
}

extern "C" mofem_status mofem_group_destroy(mofem_group g) {
    if (!g) return MOFEM_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    free_group(g);
    return MOFEM_OK;
}
