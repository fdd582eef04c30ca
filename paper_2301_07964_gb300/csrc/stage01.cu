// Stages 0 and 1 of the two-stage HT reduction on the GPU (feeders of stage 2).
//
// Stage 0: QR of B (the paper QR-factorises B before stage 1, Section "Experiments"):
//   blocked Householder QR with 32-column panels; each panel's block reflector
//   I - V T V^T is applied to the trailing columns of B, to all of A (from the left) and to Q
//   (from the right) with three GEMMs each.
// Stage 1: Alg. 1 ("Blocked stage 1") with n_b = r:
//   left: for the p*n_b x n_b blocks of the panel, bottom block first, QR of the block and
//   its block reflector applied to A(i1:i2, j2+1:n), B(i1:i2, i1:n) and Q(:, i1:i2);
//   right: for the same blocks bottom first, RQ of the filled B block, LQ of the first n_b
//   rows of its orthogonal factor (k_block_rq_lq) and the resulting block reflector applied
//   to A(:, i1:i2), B(1:i2, i1:i2) and Z(:, i1:i2); the reduced columns of the B block are
//   set to exact zeros below the diagonal.
#include "hts_internal.cuh"

namespace hts {

cudaError_t launch_panel_qr(int m, int b, double *P, int ld, double *V, int ldv, double *tau, cudaStream_t st);
cudaError_t launch_larft(int b, const double *S, int lds, const double *tau, double *T, int ldt, cudaStream_t st);
cudaError_t launch_block_rq_lq(int m, int l, const double *Bblk, int ldb, double *V, int ldv, double *tau_lq,
                               cudaStream_t st);

namespace {

constexpr int kStage0Panel = 32;

__global__ void k_zero_block_lower(double *M, int ld, int m, int l)
{
    // zero M(t+1:m-1, t) for t < l (0-based, relative to M)
    const int t = blockIdx.x;
    if (t >= l) return;
    for (int i = t + 1 + threadIdx.x; i < m; i += blockDim.x) M[(size_t)i + (size_t)t * ld] = 0.0;
}

constexpr size_t kBlasWorkspace = size_t(4) << 20;   // cuBLAS's workspace, from the caller's buffer

struct Bufs {
    double *V, *T, *S, *W, *W2, *tau;
    int ldv;
    cublasHandle_t h;
    cudaStream_t st;
};

// C := alpha op(A) op(B) + beta C, column-major, by cuBLAS on the handle's stream (a plain
// library GEMM: the WY products of the block reflectors).
cudaError_t dgemm(const Bufs &bf, bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda,
                  const double *B, int ldb, double beta, double *C, int ldc)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    const cublasStatus_t s = cublasDgemm(bf.h, ta ? CUBLAS_OP_T : CUBLAS_OP_N, tb ? CUBLAS_OP_T : CUBLAS_OP_N, M, N, K,
                                         &alpha, A, lda, B, ldb, &beta, C, ldc);
    return s == CUBLAS_STATUS_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

// The handle runs on stream st with its workspace in the caller's buffer (no allocation).
cudaError_t bind_blas(Bufs &bf, cublasHandle_t h, void *ws, cudaStream_t st)
{
    bf.h = h;
    bf.st = st;
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    // setting the stream resets the workspace, so it is set afterwards
    if (cublasSetWorkspace(h, ws, kBlasWorkspace) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    if (cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    return cudaSuccess;
}

#define CK(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) return _e; } while (0)

// T of the block reflector with vectors V (m x b)
cudaError_t form_t(const Bufs &bf, int m, int b, cudaStream_t st)
{
    CK(dgemm(bf, true, false, b, b, m, 1.0, bf.V, bf.ldv, bf.V, bf.ldv, 0.0, bf.S, b));
    return launch_larft(b, bf.S, b, bf.tau, bf.T, b, st);
}

// C (m x nc) := (I - V T V^T)^T C
cudaError_t wy_left(const Bufs &bf, int m, int b, double *C, int ldc, int nc, cudaStream_t st)
{
    if (nc <= 0) return cudaSuccess;
    CK(dgemm(bf, true, false, b, nc, m, 1.0, bf.V, bf.ldv, C, ldc, 0.0, bf.W, b));
    CK(dgemm(bf, true, false, b, nc, b, 1.0, bf.T, b, bf.W, b, 0.0, bf.W2, b));
    return dgemm(bf, false, false, m, nc, b, -1.0, bf.V, bf.ldv, bf.W2, b, 1.0, C, ldc);
}

// X (nr x m) := X (I - V T V^T)
cudaError_t wy_right(const Bufs &bf, int m, int b, double *X, int ldx, int nr, cudaStream_t st)
{
    if (nr <= 0) return cudaSuccess;
    CK(dgemm(bf, false, false, nr, b, m, 1.0, X, ldx, bf.V, bf.ldv, 0.0, bf.W, nr));
    CK(dgemm(bf, false, false, nr, b, b, 1.0, bf.W, nr, bf.T, b, 0.0, bf.W2, nr));
    return dgemm(bf, false, true, nr, m, b, -1.0, bf.W2, nr, bf.V, bf.ldv, 1.0, X, ldx);
}

}  // namespace

// Scratch of stages 0 and 1 (doubles): V (mmax x bmax), T and S (bmax x bmax), W and W2
// (n x bmax), tau (mmax).
size_t stage01_workspace_bytes(int n, int r, int p)
{
    const size_t bmax = (size_t)(r > kStage0Panel ? r : kStage0Panel);
    const size_t mmax = (size_t)(n > p * r ? n : p * r);
    const size_t dbl = mmax * bmax + 2 * bmax * bmax + 2 * (size_t)n * bmax + mmax;
    return (dbl * sizeof(double) + 255) / 256 * 256 + 6 * 256 + kBlasWorkspace;
}

static Bufs carve(void *work, int n, int r, int p)
{
    const size_t bmax = (size_t)(r > kStage0Panel ? r : kStage0Panel);
    const size_t mmax = (size_t)(n > p * r ? n : p * r);
    auto al = [](size_t x) { return (x + 31) / 32 * 32; };   // 256-byte steps in doubles
    double *w = static_cast<double *>(work);
    Bufs b;
    b.V = w; w += al(mmax * bmax);
    b.T = w; w += al(bmax * bmax);
    b.S = w; w += al(bmax * bmax);
    b.W = w; w += al((size_t)n * bmax);
    b.W2 = w; w += al((size_t)n * bmax);
    b.tau = w; w += al(mmax);
    b.ldv = (int)mmax;
    b.h = nullptr;
    b.st = nullptr;
    return b;
}

// cuBLAS's workspace: the last kBlasWorkspace bytes of the stage-0/1 scratch
static void *blas_ws(void *work, int n, int r, int p)
{
    return static_cast<char *>(work) + stage01_workspace_bytes(n, r, p) - kBlasWorkspace;
}

cudaError_t run_stage0(cublasHandle_t blas, int n, double *A, int lda, double *B, int ldb, double *Q, int ldq,
                       void *work, int r, int p, cudaStream_t st)
{
    Bufs bf = carve(work, n, r, p);
    CK(bind_blas(bf, blas, blas_ws(work, n, r, p), st));
    for (int j0 = 0; j0 < n - 1; j0 += kStage0Panel) {
        const int jb = imin(kStage0Panel, n - j0), m = n - j0;
        double *P = B + AT(ldb, j0 + 1, j0 + 1);
        bf.ldv = m;
        CK(launch_panel_qr(m, jb, P, ldb, bf.V, bf.ldv, bf.tau, st));
        CK(form_t(bf, m, jb, st));
        CK(wy_left(bf, m, jb, B + AT(ldb, j0 + 1, j0 + jb + 1), ldb, n - j0 - jb, st));
        CK(wy_left(bf, m, jb, A + AT(lda, j0 + 1, 1), lda, n, st));
        if (Q) CK(wy_right(bf, m, jb, Q + AT(ldq, 1, j0 + 1), ldq, n, st));
    }
    return cudaSuccess;
}

cudaError_t run_stage1(cublasHandle_t blas, int n, int nb, int p, double *A, int lda, double *B, int ldb, double *Q,
                       int ldq, double *Z, int ldz, void *work, cudaStream_t st)
{
    Bufs bf = carve(work, n, nb, p);
    CK(bind_blas(bf, blas, blas_ws(work, n, nb, p), st));
    for (int j = 1; j <= n - 2; j += nb) {
        const int j1 = j, j2 = imin(n, j + nb - 1), nbw = j2 - j1 + 1;
        const int num = n - nb - j + 1, den = (p - 1) * nb;
        const int nblocks = num > 0 ? (num + den - 1) / den : 0;
        // left reflectors, bottom block first
        for (int k = nblocks - 1; k >= 0; --k) {
            const int i1 = j + nb + k * (p - 1) * nb;
            const int i2 = imin(n, i1 + p * nb - 1), m = i2 - i1 + 1;
            bf.ldv = m;
            CK(launch_panel_qr(m, nbw, A + AT(lda, i1, j1), lda, bf.V, bf.ldv, bf.tau, st));
            CK(form_t(bf, m, nbw, st));
            CK(wy_left(bf, m, nbw, A + AT(lda, i1, j2 + 1), lda, n - j2, st));
            CK(wy_left(bf, m, nbw, B + AT(ldb, i1, i1), ldb, n - i1 + 1, st));
            if (Q) CK(wy_right(bf, m, nbw, Q + AT(ldq, 1, i1), ldq, n, st));
        }
        // opposite reflectors from the filled B blocks, bottom block first
        for (int k = nblocks - 1; k >= 0; --k) {
            const int i1 = j + nb + k * (p - 1) * nb;
            const int i2 = imin(n, i1 + p * nb - 1), m = i2 - i1 + 1;
            const int l = imin(nb, m);
            bf.ldv = m;
            CK(launch_block_rq_lq(m, l, B + AT(ldb, i1, i1), ldb, bf.V, bf.ldv, bf.tau, st));
            CK(form_t(bf, m, l, st));
            CK(wy_right(bf, m, l, A + AT(lda, 1, i1), lda, n, st));
            CK(wy_right(bf, m, l, B + AT(ldb, 1, i1), ldb, i2, st));
            if (Z) CK(wy_right(bf, m, l, Z + AT(ldz, 1, i1), ldz, n, st));
            k_zero_block_lower<<<l, 128, 0, st>>>(B + AT(ldb, i1, i1), ldb, m, l);
            CK(cudaGetLastError());
        }
    }
    return cudaSuccess;
}

#undef CK

}  // namespace hts
