// Internal interface between theta.cu, solve.cu and api.cpp.
#pragma once
#include "subband_ops.cuh"
#include "wdb_internal.h"

namespace wdb {

// Power iteration (Algorithm 3 step size): start vector splitmix64(seed), at most
// kPowerIters iterations, stop at relative change <= kPowerRtol; tau = 1/(kStepMargin L).
constexpr unsigned long long kPowerSeed = 12345ull;
constexpr int kPowerIters = 200;
constexpr double kPowerRtol = 1e-12;
constexpr double kStepMargin = 1.01;

// shared-memory budget of one CTA of the tiled gather engine (bytes)
constexpr int kTileSmemBudget = 32 * 1024;

template <typename T>
wdb_status th_alloc(wdb_theta* th, T** p, size_t n);
TileArgs tile_args(const wdb_theta* th, bool adj, bool fp64);
SubbandArgs subband_args(const wdb_theta* th);
RedTarget th_red(const wdb_theta* th, double* out);
bool setup_fp64(const wdb_theta* th);

wdb_status theta_build_device(wdb_theta* th, const double* psf_host, int kh, int kw, long long K, int rule,
                              cudaStream_t st);
wdb_status theta_finalize(wdb_theta* th, cudaStream_t st);
void gather_entries(const Layout& L, const std::vector<Tap>& taps, std::vector<TileEntry> (&te)[2]);
wdb_status theta_batch_plans(wdb_theta* th, cudaStream_t st);
// tiling: 0 ordinary tiles, 1 super tiles where they fit, 2 grouped items
wdb_status theta_replan(wdb_theta* th, int budget, double cap_share, double split_share, int tiling,
                        cudaStream_t st);
wdb_status theta_precond(wdb_theta* th, int kind, double eps, cudaStream_t st);
std::vector<double> precond_table(const std::vector<double>& Md, const std::vector<double>& M2d, int kind,
                                  double eps);
wdb_status precond_upload(wdb_theta* th, PrecondCache& pc, cudaStream_t st);

// Time candidate FP32 tile plans on the GPU when an operator is finalised (autotuning).
constexpr bool kAutotunePlans = true;

}  // namespace wdb
