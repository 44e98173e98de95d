// The library's own device arithmetic helpers, evaluated elementwise on device arrays
// so that tests can hold them to their definitions: the FP64 reciprocal and
// reciprocal square root from FP32 estimates, the integer-pipe binary64 <-> binary32
// conversions and tests, the double-word (float-float) split and operations, the
// exponent moves and the sign decisions of the MC and PPM limiters.  Testing only, not
// part of the paper's method; no stage kernel calls this file.
#include <cuda_runtime.h>

#include "../../include/grmhd.h"
#include "grmhd_device.cuh"

namespace grmhd {
void set_last_error(const char* msg);
}

namespace {

using namespace grmhd;

__device__ __forceinline__ double wide(float f) { return (double)f; }

// one element: in has arity(op) values, out outs(op) values
__global__ void k_numerics(int op, const double* __restrict__ in, double* __restrict__ out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        switch (op) {
        case GRMHD_NUM_RSQRT_GE1: out[i] = rsqrt_ge1(in[i]); break;
        case GRMHD_NUM_RCP_POS: out[i] = rcp_pos(in[i]); break;
        case GRMHD_NUM_D2F: out[i] = wide(d2f_int(in[i])); break;
        case GRMHD_NUM_F2D: out[i] = f2d_int(__double2float_rn(in[i])); break;
        case GRMHD_NUM_DW_SPLIT: {
            const dw x = dw_of(in[i]);
            out[2 * i] = wide(x.hi);
            out[2 * i + 1] = wide(x.lo);
            break;
        }
        case GRMHD_NUM_DW_ADD:
        case GRMHD_NUM_DW_MUL: {
            const dw a = dw_of(in[2 * i]), b = dw_of(in[2 * i + 1]);
            const dw r = op == GRMHD_NUM_DW_ADD ? dw_add(a, b) : dw_mul(a, b);
            out[2 * i] = wide(r.hi);
            out[2 * i + 1] = wide(r.lo);
            break;
        }
        case GRMHD_NUM_DW_RCP:
        case GRMHD_NUM_DW_SQRT: {
            const dw a = dw_of(in[i]);
            const dw r = op == GRMHD_NUM_DW_RCP ? dw_rcp(a) : dw_sqrt(a);
            out[2 * i] = wide(r.hi);
            out[2 * i + 1] = wide(r.lo);
            break;
        }
        case GRMHD_NUM_QUARTER: out[i] = scale_pow2<double, -2>(in[i]); break;
        case GRMHD_NUM_TWICE: out[i] = scale_pow2<double, 1>(in[i]); break;
        case GRMHD_NUM_MINMOD3: out[i] = minmod3<double>(in[3 * i], in[3 * i + 1], in[3 * i + 2]); break;
        case GRMHD_NUM_MINMOD3_F32:
            out[i] = wide(minmod3<float>(__double2float_rn(in[3 * i]), __double2float_rn(in[3 * i + 1]),
                                         __double2float_rn(in[3 * i + 2])));
            break;
        case GRMHD_NUM_PROD_SIGN:
            out[i] = prod_pos<double>(in[2 * i], in[2 * i + 1]) ? 1.0
                                                                 : (prod_neg<double>(in[2 * i], in[2 * i + 1]) ? -1.0 : 0.0);
            break;
        case GRMHD_NUM_PPM_LIMIT: {
            double aL = in[3 * i + 1], aR = in[3 * i + 2];
            ppm_limit<double>(in[3 * i], aL, aR);
            out[2 * i] = aL;
            out[2 * i + 1] = aR;
            break;
        }
        case GRMHD_NUM_TESTS: {
            const double x = in[i];
            out[i] = (finite_int(x) ? 1.0 : 0.0) + (pos_int(x) ? 2.0 : 0.0) + (mag_below_int(x, kHi1e10) ? 4.0 : 0.0);
            break;
        }
        default: break;
        }
    }
}

}  // namespace

extern "C" grmhd_status grmhd_numerics_eval(int op, const double* in, double* out, long long n,
                                            grmhd_stream_t stream)
{
    if (op < 0 || op >= GRMHD_NUM_COUNT) {
        grmhd::set_last_error("grmhd_numerics_eval: unknown op");
        return GRMHD_ERR_ARG;
    }
    if (n < 0 || (n > 0 && (!in || !out))) {
        grmhd::set_last_error("grmhd_numerics_eval: bad arguments");
        return GRMHD_ERR_ARG;
    }
    if (n == 0) return GRMHD_OK;
    const long long blocks = (n + 255) / 256;
    k_numerics<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(op, in, out, n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        grmhd::set_last_error("grmhd_numerics_eval: launch failed");
        return GRMHD_ERR_CUDA;
    }
    return GRMHD_OK;
}
