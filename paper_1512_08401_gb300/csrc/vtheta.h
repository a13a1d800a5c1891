// Internal interface of the row-varying operator (vtheta.cu): per-output-row tap plans of
// Theta_K and Theta_K^T, the construction's candidate segments, and the handle.
#pragma once
#include <vector>

#include "wdb_internal.h"

namespace wdb {

constexpr int kVTapU = 256;   // VTap.mode flag: same-level tap, ci = c - ox (mod cols)

// One output row of a plan (a subband row of the coefficient vector).
struct VRow {
    long long out_off;   // coefficient index of the row's first output
    int cols;            // outputs in the row (<= 1024)
    int sb;              // subband of the row (its weight w)
    int lgR;             // log2 of the class period 2^{J - s} along the row
    int cls_off;         // class index of the row's column 0 (preconditioner tables)
    int t0, t1;          // taps summed in registers: [t0, t1)
    int g0, g1;          // groups of coarser-input taps: [g0, g1)
};

// One tap: input row at in_off. Register taps: mode = kVTapU (ci = c - ox mod cols) or
// mode = lg r (ci = ox + r c mod r cols, input r times finer). Group taps: ci = (c - ox)/r
// for outputs c = ox (mod r), input r times coarser.
struct VTap {
    int in_off;
    int ox;
    int mode;
    int pad;
};

// Taps of one coarser input level: stride r = 2^lgr, cin input columns (cols = r cin),
// phase p's taps are [ph[ph0 + p], ph[ph0 + p + 1]).
struct VGroup {
    int lgr;
    int cin;
    int ph0;
    int pad;
};

struct VPlanDev {
    const VRow* rows = nullptr;
    const int* order = nullptr;     // rows by decreasing work (CTA i takes row order[i])
    const VTap* taps = nullptr;
    const float* v32 = nullptr;
    const double* v64 = nullptr;
    const VGroup* groups = nullptr;
    const int* ph = nullptr;
    int n_rows = 0;
};

struct VPlanHost {
    std::vector<VRow> rows;
    std::vector<int> order;
    std::vector<VTap> taps;
    std::vector<float> v32;
    std::vector<double> v64;
    std::vector<VGroup> groups;
    std::vector<int> ph;
};

// A kept tap: entries of output row (a, py) and input row (b, qy) on horizontal diagonal ox
// (column form when level(a) <= level(b): px = ox + r qx; row form: qx = ox + r px).
struct VTapH {
    int a, py, b, qy, ox;
    double v;
};

// Construction: one window of one probe's coefficients (subband sub), rows r0 + [0, h) and
// columns c0 + [0, w) (mod the subband sides), stored from candidate index base on.
struct VSeg {
    long long base;
    int sub, r0, h, c0, w;
    int kind;              // 0: column probe of (fixed_sub, fixed_row); 1: row probe
    int fixed_sub, fixed_row;
    unsigned long long mult;
    double sigma;
};

wdb_status vtheta_new(int n_rows, int n_cols, const char* wavelet, int levels, wdb_vtheta** out);
void vtheta_release(wdb_vtheta* op);
wdb_status vtheta_build_device(wdb_vtheta* op, const double* psfs_host, int kh, int kw, long long K,
                               int rule, cudaStream_t st);
wdb_status vtheta_finalize(wdb_vtheta* op, cudaStream_t st);
wdb_status vtheta_plan_emulate(const wdb_vtheta* op, bool adj, const double* x, double* y);
wdb_status vtheta_apply(const wdb_vtheta* op, const float* in, float* out, bool adj, cudaStream_t st);
wdb_status vtheta_precond(wdb_vtheta* op, int kind, double eps, cudaStream_t st);
wdb_status vtheta_set_precond(wdb_vtheta* op, int kind, const double* P, double tau);
wdb_status vtheta_objective_public(wdb_vtheta* op, const float* x, const float* x0, const double* w_host,
                                   cudaStream_t st, double* E);
wdb_status vtheta_solve(wdb_vtheta* op, const float* in, bool is_image, float* x_out,
                        const wdb_solve_params* p, cudaStream_t st, wdb_solve_result* res);

}  // namespace wdb

struct wdb_vtheta {
    wdb::Layout lay;
    wdb::Filters filt;
    std::string wavelet;
    int rule = 0;
    long long K_requested = 0, K_eff = 0, n_candidates = 0, n_cand_slots = 0;
    int n_probes = 0;
    double theta_max_abs = 0.0, build_ms = 0.0;
    std::vector<wdb::VTapH> taps;          // sorted (a, py, b, qy, ox)
    std::vector<int> cls_off;              // [S+1] class table offset of each subband
    int n_classes = 0;
    wdb::VPlanHost hplan[2];               // [0 Theta_K, 1 Theta_K^T]
    wdb::VPlanDev plan[2];
    int grid = 0;                          // CTAs of one application (rows)
    std::vector<void*> allocs;
    double* d_part = nullptr;              // grid x 3
    unsigned int* d_counter = nullptr;     // one-off reductions
    double* d_red = nullptr;               // one-off totals
    bool diag_valid = false;
    std::vector<double> Md, M2d;           // per class
    wdb::PrecondCache pc[3];
    float *d_x0 = nullptr, *d_y = nullptr, *d_r = nullptr, *d_xs = nullptr, *d_scr = nullptr, *d_w = nullptr;
    wdb::SolveState* d_state = nullptr;
    wdb::SolveState* h_state = nullptr;
    wdb::IterEngine engine[3];
    cudaStream_t work = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};
