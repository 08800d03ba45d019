// nx_runtime.h -- host-side context of libnavixgb (internal).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "navixgb.h"
#include "nx_internal.h"

struct nx_graph {
    int steps = 0;
    bool full = false;
    bool policy = false;
    bool lean = false;
    cudaGraphExec_t exec = nullptr;
};

struct nx_tune_entry {
    int group_lanes, envs_per_cta;
    float ms;
};

struct nx_env {
    // configuration
    nx_options opt{};
    uint64_t seed = 0;
    int n_envs = 0;
    int n_families = 0;
    bool rgb = false;
    bool rgb_full = false;
    std::vector<nx_desc> descs;
    std::vector<size_t> grid_offset;  // byte offset of each env's planes in the grid pool
    size_t grid_pool = 0;
    int max_side = 0;
    // slots are sized for grids of this side (<= max_side): items of larger
    // grids hold fewer envs (nx_item_envs); chosen by the autotuner
    int grid_side = 0;
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    cudaStream_t copy_stream = nullptr;

    // device memory (owned)
    std::vector<void*> allocs;
    size_t device_bytes = 0;
    nx_agent* d_agents = nullptr;
    uint8_t* d_grids = nullptr;
    nx_req* d_req = nullptr;
    nx_ctl* d_ctl = nullptr;
    uint8_t* d_atlas = nullptr;
    nx_item* d_items = nullptr;
    nx_item* d_items_fam = nullptr;
    size_t items_capacity = 0;

    // launch shape and work list
    nx_launch_shape shape{8, 32, 0};
    int n_items = 0;
    int grid_ctas = 0;
    int per_sm = 0;
    int per_sm_full = 0;  // resident CTAs of the instantiation with the fully observable views
    int lean_family = -1;  // lean step kernels: the one family of every env, or NX_N_FAMILIES (several)
    mutable int per_sm_lean = 0;  // resident CTAs of the lean instantiation (cache; 0: not queried, -1: none)
    int policy_agents = 1;        // the fused policy's weight sets per 128-env block
    std::vector<int> fam_begin;
    bool tuned = false;
    std::vector<nx_tune_entry> tune_log;
    std::vector<nx_graph> graphs;

    // fused policy (nx_set_policy): weight images, its own 128-env work list
    uint8_t* d_policy = nullptr;
    std::vector<uint8_t> policy_host;  // kept alive for the asynchronous upload
    nx_item* d_items_pol = nullptr;
    std::vector<nx_item> items_pol;
    int n_items_pol = 0;
    int per_sm_pol = 0;
    uint32_t policy_epa = 0;
    int32_t policy_shift1 = 0, policy_shift2 = 0;
    uint32_t policy_eps = 0;

    // per-call request record (host image of the fixed fields)
    nx_req req_host{};
    bool was_reset = false;

    // host-buffer rollouts
    uint8_t* host_chunk[2] = {nullptr, nullptr};
    size_t host_chunk_bytes = 0;
    cudaEvent_t ev_done[2] = {nullptr, nullptr};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};

    // instrumentation
    int64_t n_step_launches = 0;
    int64_t n_all_launches = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> prof_events;  // pool, used in pairs
    size_t prof_used = 0;

    std::string last_error;
};

nx_status nx_fail(nx_env* env, nx_status s, const std::string& msg);
nx_status nx_cuda_fail(nx_env* env, int err, const char* what);
void* nx_dev_alloc(nx_env* env, size_t bytes);
void nx_dev_free(nx_env* env, void* p);
void nx_dev_free_all(nx_env* env);
int nx_default_max_steps(int family, int size);
std::vector<nx_item> nx_build_items(const nx_env* env, const nx_launch_shape& s, int ref_side);
nx_status nx_apply_shape(nx_env* env, const nx_launch_shape& s);
void nx_drop_graphs(nx_env* env);
nx_kparams nx_params(const nx_env* env, int launch_steps, int reset_all);
nx_status nx_autotune(nx_env* env);
