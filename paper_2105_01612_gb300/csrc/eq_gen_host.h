// eq_gen_host.h - host plan of the runtime-length path (any sizes, uneven batches).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/eq.h"
#include "eq_gen.cuh"

namespace eqg {

cudaError_t gen_occupancy_f32(int kind, int threads, size_t smem, int* blocks);
cudaError_t gen_occupancy_f64(int kind, int threads, size_t smem, int* blocks);
cudaError_t gen_launch_f32(int kind, const GenArgs& a, int grid, int threads, size_t smem, cudaStream_t s);
cudaError_t gen_launch_f64(int kind, const GenArgs& a, int grid, int threads, size_t smem, cudaStream_t s);
cudaError_t gen_occupancy_dd(int kind, int threads, size_t smem, int* blocks);
cudaError_t gen_launch_dd(int kind, const GenArgs& a, int grid, int threads, size_t smem, cudaStream_t s);

struct GenPlan;

// Tunable pass shapes of the runtime-length path.
struct GenTune {
  int zc = 16, zt = 256;   // z pass: tile columns, threads per block; zc = 0 selects the
                           // warp-per-column kernel (k_gen_scols, its own block shape)
  int yc = 16, yt = 256;   // y pass, the same
  int xp = 2;              // x pass: row pairs per block (6 xp transforms, 32 threads each) of
                           // the shared-memory kernel (1..3); 0 = the warp-per-row kernel
                           // (k_gen_xrows); 4 = the warp-per-plane-pair kernel (k_gen_xpair, FP32)
};

// Largest supported axis length and the rule for it (for error messages).
bool gen_length_supported(int n);

// dims: 3 * count ints (nx, ny, nz per field); fields are packed in order in the buffers.
eq_status gen_plan_create(const int* dims, int count, eq_dtype dtype, const eq_plan_opts& o,
                          int sms, GenPlan** out, std::string* err);
// Enqueue the passes; ev (nullable) receives EQ_NUM_PASSES + 1 event records.
eq_status gen_enqueue(GenPlan* g, const void* d_in, void* d_out, cudaStream_t s, cudaEvent_t* ev,
                      std::string* err);
const eq_norms_t* gen_norms_device(const GenPlan* g);
int* gen_err_device(const GenPlan* g);     // the plan's device error word
GenTune gen_default_tune(const GenPlan* g);
eq_status gen_configure(GenPlan* g, const GenTune& t, std::string* err);
// Time candidate shapes of each pass on these buffers and keep the fastest (stored in the
// tuning cache when EQ_TUNE_CACHE names a file).
eq_status gen_autotune(GenPlan* g, const void* d_in, void* d_out, cudaStream_t s, std::string* err);
bool gen_cache_lookup(const GenPlan* g, GenTune* t);
GenTune gen_current_tune(const GenPlan* g);
size_t gen_device_bytes(const GenPlan* g);
bool gen_is_dd(const GenPlan* g);           // FP64 plan in double-float arithmetic
long long gen_total_elems(const GenPlan* g);   // 6 * sum of voxels
int gen_count(const GenPlan* g);
void gen_destroy(GenPlan* g);

}  // namespace eqg
