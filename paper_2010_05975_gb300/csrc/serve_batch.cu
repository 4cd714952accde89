// Shared launches for small solve requests (the serving runtime's batched
// path; the paper has no serving layer).  Every request of a batch is solved
// with the same kernels in one launch per step:
//   binary32 copy of A -> lu_factor_batched (Algorithm 1 per matrix, one CTA
//   each) -> x0 = LU^{-1} b -> refinement: r = b - A x (binary64), the
//   normwise backward error per column, d = LU^{-1} (r / s) s, x += d.
// A request stops refining (its `active` flag drops) as soon as its own
// backward error reaches its tolerance, so what it computes depends only on
// its own data: its result is the same alone and in any batch.
#include "common.cuh"
#include "prof.cuh"
#include <cmath>
#include <vector>

namespace lu {
namespace sb {

constexpr int kRows = 32;          // residual rows per CTA
constexpr int kRG = 8;             // right-hand sides per register group
constexpr int kJ = 128;            // columns of A staged per chunk

// n x n binary32 copy of A (ld n) for the requests that are factored here.
__global__ void convert_kernel(int batch, const BatchReq* __restrict__ rq) {
    const BatchReq& q = rq[blockIdx.y];
    if (!q.factor) return;
    const long long tot = static_cast<long long>(q.n) * q.n;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(e / q.n), c = static_cast<int>(e % q.n);
        q.F[e] = static_cast<float>(q.A[idx(r, c, q.lda)]);
    }
}

// ||A||_inf and max_i |b_ic| per column (one CTA per request).
__global__ void norms_kernel(int batch, BatchReq* __restrict__ rq) {
    BatchReq& q = rq[blockIdx.x];
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double mx = 0.0;
    for (int r = warp; r < q.n; r += nw) {
        double s = 0.0;
        for (int j = lane; j < q.n; j += 32) s += fabs(q.A[idx(r, j, q.lda)]);
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        mx = fmax(mx, s);
    }
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < nw; ++w) m = fmax(m, red[w]);
        q.anorm = m;
    }
    for (int c = threadIdx.x; c < q.nrhs; c += blockDim.x) {
        double b = 0.0;
        for (int i = 0; i < q.n; ++i) b = fmax(b, fabs(q.B[idx(i, c, q.ldb)]));
        q.cw[c] = b;                                   // cw[0 : nrhs) = bmax
    }
}

// R = B - A X for 32 rows of one request (grid.y = request).
__global__ void __launch_bounds__(256) residual_kernel(int batch, const BatchReq* __restrict__ rq,
                                                       const int* __restrict__ active) {
    const int qi = blockIdx.y;
    if (!active[qi]) return;
    const BatchReq& q = rq[qi];
    const int row0b = blockIdx.x * kRows;
    if (row0b >= q.n) return;
    __shared__ double xs[kJ][kRG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row0 = row0b + warp * 4;
    for (int g0 = 0; g0 < q.nrhs; g0 += kRG) {
        const int ng = min(kRG, q.nrhs - g0);
        double acc[4][kRG];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < kRG; ++c) acc[r][c] = 0.0;
        for (int j0 = 0; j0 < q.n; j0 += kJ) {
            __syncthreads();
            for (int e = threadIdx.x; e < kJ * kRG; e += blockDim.x) {
                const int jj = e / kRG, c = e % kRG;
                xs[jj][c] = (j0 + jj < q.n && c < ng) ? q.X[idx(j0 + jj, g0 + c, q.nrhs)] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = row0 + r;
                if (row >= q.n) continue;
                const double* arow = q.A + idx(row, j0, q.lda);
#pragma unroll
                for (int t = 0; t < kJ / 32; ++t) {
                    const int jj = lane + 32 * t;
                    const double a = (j0 + jj < q.n) ? arow[jj] : 0.0;
#pragma unroll
                    for (int c = 0; c < kRG; ++c) acc[r][c] = fma(a, xs[jj][c], acc[r][c]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < kRG; ++c) {
                double v = acc[r][c];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                acc[r][c] = v;
            }
        if (lane < kRG) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = row0 + r;
                double s = 0.0;
#pragma unroll
                for (int cc = 0; cc < kRG; ++cc)
                    if (cc == lane) s = acc[r][cc];
                if (row < q.n && lane < ng) q.R[idx(row, g0 + lane, q.nrhs)] = q.B[idx(row, g0 + lane, q.ldb)] - s;
            }
        }
    }
}

// Per column c: rmax = max|r_c|, xmax = max|x_c|, eta_c = rmax / (||A|| xmax
// + bmax); eta[request] = max_c eta_c; cw[nrhs + c] = rmax (the scale of the
// correction solve).  One CTA per request, one warp per column.
__global__ void eta_kernel(int batch, const BatchReq* __restrict__ rq, const int* __restrict__ active,
                           double* __restrict__ eta) {
    const int qi = blockIdx.x;
    if (!active[qi]) return;
    const BatchReq& q = rq[qi];
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double em = 0.0;
    for (int c = warp; c < q.nrhs; c += nw) {
        double rm = 0.0, xm = 0.0;
        for (int i = lane; i < q.n; i += 32) {
            rm = fmax(rm, fabs(q.R[idx(i, c, q.nrhs)]));
            xm = fmax(xm, fabs(q.X[idx(i, c, q.nrhs)]));
        }
        for (int off = 16; off > 0; off >>= 1) {
            rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, off));
            xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, off));
        }
        const double den = q.anorm * xm + q.cw[c];
        em = fmax(em, den > 0.0 ? rm / den : 0.0);
        if (lane == 0) q.cw[q.nrhs + c] = rm;
    }
    if (lane == 0) red[warp] = em;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < nw; ++w) m = fmax(m, red[w]);
        eta[qi] = m;
    }
}

// r = src / s_c in binary32 (src = B with s = bmax for x0, else R with s = rmax).
__global__ void scale_kernel(int batch, const BatchReq* __restrict__ rq, const int* __restrict__ active, int from_b) {
    const int qi = blockIdx.y;
    if (!active[qi]) return;
    const BatchReq& q = rq[qi];
    const long long tot = static_cast<long long>(q.n) * q.nrhs;
    const double* sc = q.cw + (from_b ? 0 : q.nrhs);
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(e / q.nrhs), c = static_cast<int>(e % q.nrhs);
        const double v = from_b ? q.B[idx(i, c, q.ldb)] : q.R[e];
        q.r[e] = static_cast<float>(sc[c] > 0.0 ? v / sc[c] : 0.0);
    }
}

// r := U^{-1} L^{-1} P r with the binary32 factors, one CTA per request, one
// warp per right-hand side (groups of 8).
__global__ void __launch_bounds__(256) solve_kernel(int batch, const BatchReq* __restrict__ rq,
                                                    const int* __restrict__ active) {
    const int qi = blockIdx.x;
    if (!active[qi]) return;
    const BatchReq& q = rq[qi];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* ybuf = reinterpret_cast<float*>(smem_raw);    // 8 x n
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = q.n;
    for (int c0 = 0; c0 < q.nrhs; c0 += 8) {
        const int col = c0 + warp;
        if (col < q.nrhs) {
            float* yc = ybuf + static_cast<size_t>(warp) * n;
            for (int i = lane; i < n; i += 32) yc[i] = q.r[idx(i, col, q.nrhs)];
            __syncwarp();
            if (lane == 0)
                for (int i = 0; i < n; ++i) {
                    const int p = q.piv[i];
                    const float t = yc[i];
                    yc[i] = yc[p];
                    yc[p] = t;
                }
            __syncwarp();
            for (int i = 1; i < n; ++i) {                // forward, unit L
                float s = 0.f;
                for (int p = lane; p < i; p += 32) s = fmaf(q.F[idx(i, p, n)], yc[p], s);
                for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                if (lane == 0) yc[i] -= s;
                __syncwarp();
            }
            for (int i = n - 1; i >= 0; --i) {           // backward, U
                float s = 0.f;
                for (int p = i + 1 + lane; p < n; p += 32) s = fmaf(q.F[idx(i, p, n)], yc[p], s);
                for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                if (lane == 0) yc[i] = (yc[i] - s) / q.F[idx(i, i, n)];
                __syncwarp();
            }
            for (int i = lane; i < n; i += 32) q.r[idx(i, col, q.nrhs)] = yc[i];
        }
        __syncthreads();
    }
}

// X = (set ? 0 : X) + s_c r   (binary64)
__global__ void update_kernel(int batch, const BatchReq* __restrict__ rq, const int* __restrict__ active, int set) {
    const int qi = blockIdx.y;
    if (!active[qi]) return;
    const BatchReq& q = rq[qi];
    const long long tot = static_cast<long long>(q.n) * q.nrhs;
    const double* sc = q.cw + (set ? 0 : q.nrhs);
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < tot;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(e % q.nrhs);
        const double d = static_cast<double>(q.r[e]) * sc[c];
        q.X[e] = set ? d : q.X[e] + d;
    }
}

}  // namespace sb

extern "C" int lu_factor_batched(int batch, const int* n, void* const* A, const int* lda, int* const* piv, int* info,
                                 int dtype, cudaStream_t stream);

// Solve every request of the batch (see the file comment).  `h` holds the
// requests on the host (device pointers inside); tol[i] is request i's
// target.  On return out[i] is 0 (converged: iters[i] refinement steps,
// eta[i]), 1 (singular factor: info != 0), or 2 (stopped contracting before
// tol: the request needs a stronger solver).  Returns 0 or LU_E*.
int batch_solve(std::vector<BatchReq>& h, const std::vector<double>& tol, int max_iter, std::vector<int>& out,
                std::vector<int>& iters, std::vector<double>& eta_out, cudaStream_t s) {
    const int nb = static_cast<int>(h.size());
    out.assign(nb, 0);
    iters.assign(nb, 0);
    eta_out.assign(nb, 0.0);
    if (nb == 0) return 0;
    int nmax = 0, rmax = 0, nf = 0;
    for (const BatchReq& q : h) {
        nmax = q.n > nmax ? q.n : nmax;
        rmax = q.nrhs > rmax ? q.nrhs : rmax;
        nf += q.factor;
    }
    // device: requests, active flags, eta, and the factor launch's arrays
    const size_t bytes = sizeof(BatchReq) * nb + sizeof(int) * nb + sizeof(double) * nb +
                         (sizeof(void*) * 2 + sizeof(int) * 3) * static_cast<size_t>(nf > 0 ? nf : 1) + 256;
    unsigned char* ws = nullptr;
    if (lu_malloc_async(reinterpret_cast<void**>(&ws), bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return LU_ENOMEM;
    }
    BatchReq* drq = reinterpret_cast<BatchReq*>(ws);
    double* deta = reinterpret_cast<double*>(drq + nb);
    void** fA = reinterpret_cast<void**>(deta + nb);
    int** fP = reinterpret_cast<int**>(fA + (nf > 0 ? nf : 1));
    int* act = reinterpret_cast<int*>(fP + (nf > 0 ? nf : 1));
    int* fn = act + nb;
    int* fld = fn + (nf > 0 ? nf : 1);
    int* finfo = fld + (nf > 0 ? nf : 1);
    std::vector<void*> hA;
    std::vector<int*> hP;
    std::vector<int> hn, hld, fidx;
    for (int i = 0; i < nb; ++i)
        if (h[i].factor) {
            hA.push_back(h[i].F);
            hP.push_back(h[i].piv);
            hn.push_back(h[i].n);
            hld.push_back(h[i].n);
            fidx.push_back(i);
        }
    std::vector<int> active(nb, 1), info(nf > 0 ? nf : 1, 0);
    std::vector<double> eta(nb, 0.0), prev(nb, 0.0);
    std::vector<int> slow(nb, 0);
    int rc = 0;
    const int gy = nb;
    auto fail = [&](int r) { rc = r; };
    if (cudaMemcpyAsync(drq, h.data(), sizeof(BatchReq) * nb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(act, active.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s) != cudaSuccess)
        fail(LU_ELAUNCH);
    if (!rc && nf > 0 &&
        (cudaMemcpyAsync(fA, hA.data(), sizeof(void*) * nf, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(fP, hP.data(), sizeof(int*) * nf, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(fn, hn.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(fld, hld.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, s) != cudaSuccess))
        fail(LU_ELAUNCH);
    const int gx_elem = cdiv(static_cast<int>(std::min<long long>(static_cast<long long>(nmax) * nmax, 1 << 22)), 256 * 4);
    const int gx_vec = cdiv(nmax * rmax, 256) > 0 ? cdiv(nmax * rmax, 256) : 1;
    if (!rc) {
        ProfScope ps(LU_PROF_OTHER, s);
        sb::convert_kernel<<<dim3(gx_elem > 0 ? gx_elem : 1, gy), 256, 0, s>>>(nb, drq);
        sb::norms_kernel<<<nb, 256, 0, s>>>(nb, drq);
        count_launches(2);
        if (cudaPeekAtLastError() != cudaSuccess) fail(LU_ELAUNCH);
    }
    if (!rc && nf > 0) rc = lu_factor_batched(nf, fn, fA, fld, fP, finfo, LU_PREC_F32, s);
    const size_t ssmem = 8 * static_cast<size_t>(nmax > 0 ? nmax : 1) * sizeof(float);
    if (!rc) rc = smem_attr(sb::solve_kernel, ssmem);
    auto correction = [&](int from_b) {
        {
            ProfScope ps(LU_PROF_OTHER, s);
            sb::scale_kernel<<<dim3(gx_vec, gy), 256, 0, s>>>(nb, drq, act, from_b);
            count_launches(1);
        }
        {
            ProfScope ps(LU_PROF_SOLVE, s);
            sb::solve_kernel<<<nb, 256, ssmem, s>>>(nb, drq, act);
            count_launches(1);
        }
        {
            ProfScope ps(LU_PROF_OTHER, s);
            sb::update_kernel<<<dim3(gx_vec, gy), 256, 0, s>>>(nb, drq, act, from_b);
            count_launches(1);
        }
        if (cudaPeekAtLastError() != cudaSuccess) fail(LU_ELAUNCH);
    };
    // factorization status: singular requests stop here
    if (!rc && nf > 0) {
        if (cudaMemcpyAsync(info.data(), finfo, sizeof(int) * nf, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            fail(LU_ELAUNCH);
        bool change = false;
        for (int j = 0; j < nf && !rc; ++j)
            if (info[j] != 0) {
                out[fidx[j]] = 1;
                active[fidx[j]] = 0;
                change = true;
            }
        if (change && cudaMemcpyAsync(act, active.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s) != cudaSuccess)
            fail(LU_ELAUNCH);
    }
    if (!rc) correction(1);                               // x0 = LU^{-1} b
    for (int it = 0; !rc; ++it) {
        {
            ProfScope ps(LU_PROF_RESIDUAL, s);
            sb::residual_kernel<<<dim3(cdiv(nmax, sb::kRows), gy), 256, 0, s>>>(nb, drq, act);
            sb::eta_kernel<<<nb, 256, 0, s>>>(nb, drq, act, deta);
            count_launches(2);
        }
        if (cudaPeekAtLastError() != cudaSuccess ||
            cudaMemcpyAsync(eta.data(), deta, sizeof(double) * nb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            fail(LU_ELAUNCH);
            break;
        }
        int left = 0;
        for (int i = 0; i < nb; ++i) {
            if (!active[i]) continue;
            eta_out[i] = eta[i];
            iters[i] = it;
            if (eta[i] <= tol[i]) {
                active[i] = 0;                            // converged: frozen from here on
                continue;
            }
            // classical refinement must keep contracting: two steps that do
            // not halve the error, or max_iter steps, hand the request on
            if (it > 0 && eta[i] > 0.5 * prev[i]) ++slow[i];
            if (slow[i] >= 2 || it >= max_iter) {
                active[i] = 0;
                out[i] = 2;
                continue;
            }
            prev[i] = eta[i];
            ++left;
        }
        if (!left) break;
        if (cudaMemcpyAsync(act, active.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            fail(LU_ELAUNCH);
            break;
        }
        correction(0);
    }
    cudaGetLastError();
    cudaFreeAsync(ws, s);
    return rc;
}

}  // namespace lu
