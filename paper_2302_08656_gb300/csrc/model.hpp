// The GPU model of an ACOPF instance (model.cu: KKT pattern and assembly;
// ipm.cu: the interior-point loop's data and workspace).
#pragma once
#include <cstdint>
#include <vector>

struct kkt_model {
    int nb = 0, nl = 0, ng = 0, flow = 0;
    int n_primal = 0, n = 0;
    int64_t nnz = 0;
    std::vector<int> rowptr, colidx;     // host copy of the pattern
    std::vector<int> from, to, gen_bus;  // host copy of the topology
    std::vector<double> c2;
    char* base = nullptr;                // one device allocation
    int *d_f = nullptr, *d_t = nullptr, *d_tptr = nullptr, *d_tidx = nullptr, *d_kind = nullptr, *d_arg = nullptr;
    double *d_g = nullptr, *d_b = nullptr, *d_twoc2 = nullptr, *d_terms = nullptr;
    // interior-point loop (kkt_model_set_limits): loads, bounds, limits,
    // topology lists and the loop's workspace, in one device allocation
    char* ipm_base = nullptr;
    double* ipm_pin = nullptr;           // pinned mirror of the loop's scalars
    double *d_Pd = nullptr, *d_Qd = nullptr, *d_lo = nullptr, *d_hi = nullptr, *d_u = nullptr;
    int *d_bus_ptr = nullptr, *d_bus_end = nullptr, *d_gen_of_bus = nullptr, *d_rowptr = nullptr, *d_colidx = nullptr;
    double *d_s = nullptr, *d_w = nullptr, *d_zL = nullptr, *d_zU = nullptr;
    double *d_PQ = nullptr, *d_cE = nullptr, *d_cI = nullptr, *d_sigma = nullptr, *d_D = nullptr, *d_vals = nullptr;
    double *d_jtl = nullptr, *d_rhs = nullptr, *d_dir = nullptr, *d_dzL = nullptr, *d_dzU = nullptr, *d_ds = nullptr;
    double *d_dw = nullptr, *d_red = nullptr;
};
