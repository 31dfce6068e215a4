// pairs_tc.cuh -- tcgen05 all-pairs kernels (placeholder until the tensor path lands).
#pragma once
#include <string>

#include "common.cuh"

namespace clusco {

struct TcArgs {
    int form;
    void *planes;
    float *scales;
    double *G64;
    float *G32;
    int64_t N, L, Lp, Rpad, row_begin, row_end;
    float *out;
    int64_t out_base;
};

inline int tc_supported(int form, int64_t L)
{
    (void)form;
    (void)L;
    return CLUSCO_EUNSUPPORTED;
}

inline int tc_launch_allpairs(const TcArgs &a, cudaStream_t st, std::string &err)
{
    (void)a;
    (void)st;
    err = "tensor-core forms not built";
    return CLUSCO_EUNSUPPORTED;
}

}  // namespace clusco
