/*
 * FP64 CPU oracle for the HOSCF all-pairs TTVc (tensor-times-vector chain).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
 * reference legs load it.  It shares no code, header or table with the CUDA
 * library under paper_2403_01778_gb300/csrc.
 *
 * Every routine is the plain definition from the paper, written as nested
 * loops with FP64 accumulation and no blocking, fusion or reordering:
 *
 *   Sec. 2, TTV / TTVc definitions:
 *       [A x_n v]_{..i_{n-1} i_{n+1}..} = sum_{i_n} A_{i_1..i_d} v_{i_n}
 *   Eq. (3.3), coupling block of the NEPv map (3.2):
 *       A_{m,n}(x) = A x_{k != m,n} u^(k)      (an I_m x I_n matrix)
 *   Eq. (2.4), KKT left-hand sides:
 *       g_n = A x_{k != n} u^(k)   (one vector per mode)
 *
 * Conventions (fixed by this build, stated here so the file stands alone):
 *   - the tensor is row-major, last index fastest (flat index
 *     i_1*I_2*...*I_d + ... + i_d, 0-based);
 *   - the factor vectors u^(1..d) are concatenated into one array, mode n
 *     starting at offset I_1+...+I_{n-1};
 *   - the blocks A_{m,n} for m < n are packed in lexicographic (m,n) order,
 *     each row-major I_m x I_n.
 *
 * Element types accepted for the tensor: 0 = float32, 1 = float64.
 * Threads: nthreads <= 0 means "OpenMP default"; the flat index range is split
 * across threads, each with private FP64 accumulators that are summed at the
 * end (only the rounding order differs from the serial loop).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define REF_MAX_ORDER 16

static double elem(const void* T, int dtype, int64_t i) {
    if (dtype == 0) return (double)((const float*)T)[i];
    return ((const double*)T)[i];
}

static void decode(int64_t flat, int d, const int64_t* dims, int64_t* idx) {
    for (int k = d - 1; k >= 0; --k) {
        idx[k] = flat % dims[k];
        flat /= dims[k];
    }
}

static int64_t numel(int d, const int64_t* dims) {
    int64_t n = 1;
    for (int k = 0; k < d; ++k) n *= dims[k];
    return n;
}

static void mode_offsets(int d, const int64_t* dims, int64_t* off) {
    off[0] = 0;
    for (int k = 1; k < d; ++k) off[k] = off[k - 1] + dims[k - 1];
}

/* Offsets of the packed blocks (m<n, lexicographic); returns total size P. */
int64_t ref_block_offsets(int d, const int64_t* dims, int64_t* boff) {
    int64_t p = 0;
    int b = 0;
    for (int m = 0; m < d; ++m)
        for (int n = m + 1; n < d; ++n) {
            boff[b++] = p;
            p += dims[m] * dims[n];
        }
    return p;
}

static int check_args(int d, const int64_t* dims) {
    if (d < 2 || d > REF_MAX_ORDER) return -1;
    for (int k = 0; k < d; ++k)
        if (dims[k] < 1) return -1;
    return 0;
}

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) return nthreads;
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/*
 * All coupling blocks, eq. (3.3), by their definition: every element of the
 * tensor contributes T[i] * prod_{k != m,n} u^(k)[i_k] to entry (i_m, i_n) of
 * block (m, n), for every pair m < n.  H (P doubles) is overwritten.
 */
int ref_blocks(const void* T, int dtype, int d, const int64_t* dims,
               const double* u, double* H, int nthreads) {
    if (check_args(d, dims)) return -1;
    int64_t off[REF_MAX_ORDER], boff[REF_MAX_ORDER * REF_MAX_ORDER];
    mode_offsets(d, dims, off);
    int64_t P = ref_block_offsets(d, dims, boff);
    int64_t N = numel(d, dims);
    int nt = set_threads(nthreads);
    double* acc = (double*)calloc((size_t)nt * (size_t)P, sizeof(double));
    if (!acc) return -2;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* h = acc + (size_t)tid * (size_t)P;
        int64_t idx[REF_MAX_ORDER];
        int64_t lo = N * tid / nt, hi = N * (tid + 1) / nt;
        for (int64_t flat = lo; flat < hi; ++flat) {
            decode(flat, d, dims, idx);
            double t = elem(T, dtype, flat);
            int b = 0;
            for (int m = 0; m < d; ++m)
                for (int n = m + 1; n < d; ++n, ++b) {
                    double p = t;
                    for (int k = 0; k < d; ++k)
                        if (k != m && k != n) p *= u[off[k] + idx[k]];
                    h[boff[b] + idx[m] * dims[n] + idx[n]] += p;
                }
        }
    }
    for (int64_t q = 0; q < P; ++q) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += acc[(size_t)t * (size_t)P + q];
        H[q] = s;
    }
    free(acc);
    return 0;
}

/*
 * One entry of one block, eq. (3.3): A_{m,n}[i, j] summed over every
 * multi-index with i_m = i and i_n = j.  Used to check single outputs of
 * tensors too large for ref_blocks.
 */
int ref_block_entry(const void* T, int dtype, int d, const int64_t* dims,
                    const double* u, int m, int n, int64_t i, int64_t j,
                    double* out) {
    if (check_args(d, dims) || m < 0 || n >= d || m >= n) return -1;
    if (i < 0 || i >= dims[m] || j < 0 || j >= dims[n]) return -1;
    int64_t off[REF_MAX_ORDER];
    mode_offsets(d, dims, off);
    int64_t N = numel(d, dims);
    int64_t idx[REF_MAX_ORDER];
    double s = 0.0;
    for (int64_t flat = 0; flat < N; ++flat) {
        decode(flat, d, dims, idx);
        if (idx[m] != i || idx[n] != j) continue;
        double p = elem(T, dtype, flat);
        for (int k = 0; k < d; ++k)
            if (k != m && k != n) p *= u[off[k] + idx[k]];
        s += p;
    }
    *out = s;
    return 0;
}

/*
 * Strided variant of ref_block_entry that visits only the multi-indices with
 * i_m = i and i_n = j (same sum, same order of terms as the flat scan), so one
 * entry of a 1024^3 tensor costs 1024 terms instead of 2^30 index decodes.
 */
int ref_block_entry_fast(const void* T, int dtype, int d, const int64_t* dims,
                         const double* u, int m, int n, int64_t i, int64_t j,
                         double* out) {
    if (check_args(d, dims) || m < 0 || n >= d || m >= n) return -1;
    if (i < 0 || i >= dims[m] || j < 0 || j >= dims[n]) return -1;
    int64_t off[REF_MAX_ORDER], stride[REF_MAX_ORDER];
    mode_offsets(d, dims, off);
    stride[d - 1] = 1;
    for (int k = d - 2; k >= 0; --k) stride[k] = stride[k + 1] * dims[k + 1];
    int64_t M = numel(d, dims) / (dims[m] * dims[n]);
    int64_t idx[REF_MAX_ORDER];
    double s = 0.0;
    for (int64_t r = 0; r < M; ++r) {
        /* decode r over the modes other than m, n (row-major order) */
        int64_t rr = r;
        for (int k = d - 1; k >= 0; --k) {
            if (k == m || k == n) continue;
            idx[k] = rr % dims[k];
            rr /= dims[k];
        }
        idx[m] = i;
        idx[n] = j;
        int64_t flat = 0;
        for (int k = 0; k < d; ++k) flat += idx[k] * stride[k];
        double p = elem(T, dtype, flat);
        for (int k = 0; k < d; ++k)
            if (k != m && k != n) p *= u[off[k] + idx[k]];
        s += p;
    }
    *out = s;
    return 0;
}

/*
 * KKT left-hand sides, eq. (2.4): g_n = A x_{k != n} u^(k) for every mode n,
 * computed straight from the tensor (not from the blocks).  g has sum_n I_n
 * doubles, laid out like u.  Also returns the full contraction
 * A x_1 u^(1) ... x_d u^(d) in *full (the last line of (2.4)).
 */
int ref_kkt_vectors(const void* T, int dtype, int d, const int64_t* dims,
                    const double* u, double* g, double* full, int nthreads) {
    if (check_args(d, dims)) return -1;
    int64_t off[REF_MAX_ORDER];
    mode_offsets(d, dims, off);
    int64_t n_tot = off[d - 1] + dims[d - 1];
    int64_t N = numel(d, dims);
    int nt = set_threads(nthreads);
    double* acc = (double*)calloc((size_t)nt * (size_t)(n_tot + 1), sizeof(double));
    if (!acc) return -2;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* h = acc + (size_t)tid * (size_t)(n_tot + 1);
        int64_t idx[REF_MAX_ORDER];
        int64_t lo = N * tid / nt, hi = N * (tid + 1) / nt;
        for (int64_t flat = lo; flat < hi; ++flat) {
            decode(flat, d, dims, idx);
            double t = elem(T, dtype, flat);
            double all = t;
            for (int k = 0; k < d; ++k) all *= u[off[k] + idx[k]];
            h[n_tot] += all;
            for (int n = 0; n < d; ++n) {
                double p = t;
                for (int k = 0; k < d; ++k)
                    if (k != n) p *= u[off[k] + idx[k]];
                h[off[n] + idx[n]] += p;
            }
        }
    }
    for (int64_t q = 0; q <= n_tot; ++q) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += acc[(size_t)t * (size_t)(n_tot + 1) + q];
        if (q < n_tot) g[q] = s; else *full = s;
    }
    free(acc);
    return 0;
}

/*
 * Tensor-times-vector along one mode (Sec. 2 definition):
 * out = A x_n v, an order-(d-1) tensor in row-major order of the remaining
 * modes.  Used by the HOPM cross-check.
 */
int ref_ttv(const void* T, int dtype, int d, const int64_t* dims, int n,
            const double* v, double* out) {
    if (check_args(d, dims) || n < 0 || n >= d) return -1;
    int64_t N = numel(d, dims);
    int64_t M = N / dims[n];
    memset(out, 0, (size_t)M * sizeof(double));
    int64_t idx[REF_MAX_ORDER];
    for (int64_t flat = 0; flat < N; ++flat) {
        decode(flat, d, dims, idx);
        int64_t o = 0;
        for (int k = 0; k < d; ++k) {
            if (k == n) continue;
            o = o * dims[k] + idx[k];
        }
        out[o] += elem(T, dtype, flat) * v[idx[n]];
    }
    return 0;
}

/*
 * Gradient write for the adjoint of the rank-one solution (no counterpart in
 * the paper; the formula is the envelope theorem plus the implicit-function
 * adjoint): out[i] = c * prod_k u^(k)[i_k]
 *                    - sum_n a^(n)[i_n] * prod_{k != n} u^(k)[i_k]
 * with a laid out like u.
 */
int ref_grad_tensor(int d, const int64_t* dims, const double* u,
                    const double* a, double c, double* out) {
    if (check_args(d, dims)) return -1;
    int64_t off[REF_MAX_ORDER];
    mode_offsets(d, dims, off);
    int64_t N = numel(d, dims);
    int64_t idx[REF_MAX_ORDER];
    for (int64_t flat = 0; flat < N; ++flat) {
        decode(flat, d, dims, idx);
        double all = c;
        for (int k = 0; k < d; ++k) all *= u[off[k] + idx[k]];
        double s = all;
        for (int n = 0; n < d; ++n) {
            double p = a[off[n] + idx[n]];
            for (int k = 0; k < d; ++k)
                if (k != n) p *= u[off[k] + idx[k]];
            s -= p;
        }
        out[flat] = s;
    }
    return 0;
}
