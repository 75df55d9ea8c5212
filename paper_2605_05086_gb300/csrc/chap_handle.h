// The handle behind struct chap_bs (shared by the C ABI files).
#pragma once
#include "../../include/chap.h"
#include "chap_internal.h"

#include <cstdint>
#include <string>
#include <vector>

struct chap_bs {
    using Dev = chap::Dev;
    using LaunchPlan = chap::LaunchPlan;
    using Ctl = chap::Ctl;
    cudaStream_t st = nullptr;
    cudaStream_t cap_st = nullptr;
    chap_options opt{};
    chap_info info{};
    int n = 0, m = 0, m_norm = 0;
    std::vector<double> lb, ub, obj;
    std::vector<uint8_t> vtype, row_eq;
    std::vector<uint8_t> row_int, row_le;   // integral rows; rows given as "<=" (cutoff candidates)
    std::vector<int> nrow_base;
    std::vector<void *> allocs;
    Dev dev{};
    LaunchPlan plan{};
    // device scratch for host-memory outputs
    double *t_xhat = nullptr;
    long long *t_s = nullptr;
    int *t_dc = nullptr;
    int *t_w = nullptr;
    double *t_r = nullptr;
    long long *t_tabu = nullptr;
    Ctl *h_ctl = nullptr;  // pinned
    cudaGraphExec_t gexec = nullptr;
    int g_iters = 0;
    bool broken = false;
    bool prof_valid = false;   // a pass ran with kernel timing since it was enabled
    chap_move_record *t_rec = nullptr;  // move records staged from host memory
    double *t_obj = nullptr;            // objective value and the partial sums of its reduction (1 + 128)
    int shard_rank = 0, shard_count = 1;  // column shard evaluated by this handle
    int64_t hist_bins = 0;     // counting-sort bins of the instance
    bool no_hist_scratch = false; // created without the counting-sort scratch (static_scratch_only)
    long fail_allocs_after = -1; // device allocations left before an injected failure (-1: none)
    void *learn = nullptr;     // state of the learned driver (learned.cu), created on first use
    std::string err;
};

namespace chap {
// A best-shift pass (evaluation kernels + selection) on the handle's stream,
// with optional device per-variable outputs; the apply of the selected move.
cudaError_t bs_pass(chap_bs *h, const VarOut &o);
cudaError_t bs_apply_selected(chap_bs *h);
// CHAP_OK when the handle may run a pass on its own scratch; CHAP_E_STATE (with
// the handle's message set) when it was created without the counting-sort
// scratch and the instance has counting-sorted columns.
chap_status own_scratch_ok(chap_bs *h);
// CHAP_OK unless the handle evaluates only a column shard (then a pass gives
// the shard's best move, not the instance's: CHAP_E_STATE with a message).
chap_status whole_instance_ok(chap_bs *h);
constexpr int kMaxRecords = 1024;   // move records one chap_bs_apply_records call reduces
void learn_free(chap_bs *h);   // releases h->learn (learned.cu)
}  // namespace chap
