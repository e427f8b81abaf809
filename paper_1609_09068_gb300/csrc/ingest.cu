// ingest.cu -- graph model of Sec. 3 and Def. 3.4: validate the CSR (simple
// digraph: sorted, duplicate-free rows), drop self-loops (Sec. 4.1 and 5.2
// ignore them), out-degree without loops, and the in-adjacency (CSC) with
// sources ascending inside each column (stable radix sort by target).
#include "common.cuh"
#include "spmv.cuh"

namespace prgb {

// one warp per row: range and order checks, loop detection, loop-free degree
__global__ void validate_rows_k(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                int32_t n, int64_t nnz, int32_t* __restrict__ outdeg,
                                uint8_t* __restrict__ has_loop, Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const int64_t s = rowptr[i], e = rowptr[i + 1];
    bool bad = (s > e) || (s < 0) || (e > nnz) || (i == 0 && s != 0) || (i == n - 1 && e != nnz);
    int loop = 0;
    if (!bad) {
      for (int64_t k = s + lane; k < e; k += 32) {
        const int32_t c = col[k];
        if (c < 0 || c >= n) bad = true;
        if (k > s && col[k - 1] >= c) bad = true;
        if (c == (int32_t)i) loop = 1;
      }
    }
    bad = __any_sync(0xffffffffu, bad);
    loop = __any_sync(0xffffffffu, loop);
    if (lane == 0) {
      if (bad) set_err(ctl, PR_EINVAL, 1);
      outdeg[i] = bad ? 0 : (int32_t)(e - s) - loop;
      has_loop[i] = (uint8_t)loop;
    }
  }
}

// copy non-loop entries; also records the source row of every kept edge
__global__ void strip_loops_k(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              int32_t n, const uint8_t* __restrict__ has_loop,
                              const int32_t* __restrict__ optr, int32_t* __restrict__ oidx,
                              uint32_t* __restrict__ key_dst, uint32_t* __restrict__ val_src,
                              int32_t* __restrict__ indeg) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const int64_t s = rowptr[i], e = rowptr[i + 1];
    const int64_t o = optr[i];
    const bool lp = has_loop[i] != 0;
    for (int64_t k = s + lane; k < e; k += 32) {
      const int32_t c = col[k];
      if (c == (int32_t)i) continue;
      const int64_t pos = o + (k - s) - ((lp && c > (int32_t)i) ? 1 : 0);
      oidx[pos] = c;
      key_dst[pos] = (uint32_t)c;
      val_src[pos] = (uint32_t)i;
      atomicAdd(&indeg[c], 1);
    }
  }
}

static unsigned grid_rows(int64_t n) {
  int64_t warps_per_block = kBlock / 32;
  int64_t g = (n + warps_per_block - 1) / warps_per_block;
  int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

pr_status ingest(const pr_csr* csr, DevGraph* g, Arena& keep, Arena& tmp, Ctl* ctl) {
  cudaStream_t s = tmp.stream();
  const int32_t n = csr->n;
  const int64_t nnz = csr->nnz;
  g->n = n;
  const int32_t* rowptr = csr->rowptr;
  const int32_t* col = csr->col;
  if (csr->on_host) {
    int32_t *drp = nullptr, *dcol = nullptr;
    PRGB_TRY(tmp.alloc(&drp, (size_t)n + 1));
    PRGB_TRY(tmp.alloc(&dcol, (size_t)(nnz > 0 ? nnz : 1)));
    PRGB_CUDA(cudaMemcpyAsync(drp, rowptr, ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, s));
    if (nnz > 0) PRGB_CUDA(cudaMemcpyAsync(dcol, col, (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
    rowptr = drp;
    col = dcol;
  }
  PRGB_TRY(keep.alloc(&g->outdeg, (size_t)n + 1));
  PRGB_TRY(keep.alloc(&g->optr, (size_t)n + 1));
  PRGB_TRY(keep.alloc(&g->iptr, (size_t)n + 1));
  uint8_t* has_loop = nullptr;
  PRGB_TRY(tmp.alloc(&has_loop, (size_t)n + 1));
  if (n > 0) {
    validate_rows_k<<<grid_rows(n), kBlock, 0, s>>>(rowptr, col, n, nnz, g->outdeg, has_loop, ctl);
    PRGB_LAUNCH();
  }
  PRGB_TRY(scan_i32(g->outdeg, g->optr, n, tmp));
  // the loop-free edge count and the validation verdict are needed on the host
  int32_t m32 = 0;
  int err = 0;
  PRGB_CUDA(cudaMemcpyAsync(&m32, g->optr + n, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaMemcpyAsync(&err, &ctl->err, 4, cudaMemcpyDeviceToHost, s));
  PRGB_CUDA(cudaStreamSynchronize(s));
  if (err) return (pr_status)err;
  g->m = m32;
  const int64_t m = g->m;
  PRGB_TRY(keep.alloc(&g->oidx, (size_t)(m > 0 ? m : 1)));
  PRGB_TRY(keep.alloc(&g->iidx, (size_t)(m > 0 ? m : 1)));
  uint32_t *kd = nullptr, *vs = nullptr, *kt = nullptr, *vt = nullptr;
  int32_t* indeg = nullptr;
  PRGB_TRY(tmp.alloc(&kd, (size_t)(m > 0 ? m : 1)));
  PRGB_TRY(tmp.alloc(&vs, (size_t)(m > 0 ? m : 1)));
  PRGB_TRY(tmp.alloc(&kt, (size_t)(m > 0 ? m : 1)));
  PRGB_TRY(tmp.alloc(&vt, (size_t)(m > 0 ? m : 1)));
  PRGB_TRY(tmp.alloc(&indeg, (size_t)n + 1));
  PRGB_CUDA(cudaMemsetAsync(indeg, 0, ((size_t)n + 1) * 4, s));
  if (n > 0) {
    strip_loops_k<<<grid_rows(n), kBlock, 0, s>>>(rowptr, col, n, has_loop, g->optr, g->oidx, kd, vs, indeg);
    PRGB_LAUNCH();
  }
  PRGB_TRY(scan_i32(indeg, g->iptr, n, tmp));
  // CSR order is (source asc, target asc); a stable sort by target gives
  // each column's sources in ascending order.
  PRGB_TRY(radix_sort_pairs(kd, vs, kt, vt, m, bits_for((uint32_t)(n > 0 ? n - 1 : 0)), tmp));
  if (m > 0) PRGB_CUDA(cudaMemcpyAsync(g->iidx, vs, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
  PRGB_TRY(build_heavy(g->iptr, n, keep, tmp, &g->heavy_rows, &g->heavy_choff, &g->heavy_chrow, &g->nheavy,
                        &g->nchunks));
  PRGB_TRY(build_lorder(g->iptr, n, nullptr, 0, keep, tmp, &g->lorder));
  PRGB_TRY(build_lpre(g->iptr, g->lorder, n, g->m, keep, tmp, &g->lpre));
  {
    // vertices with many out-edges: the partitioner gives them a warp each
    int32_t *choff = nullptr, *chrow = nullptr, nch = 0;
    PRGB_TRY(build_heavy(g->optr, n, keep, tmp, &g->oheavy, &choff, &chrow, &g->noheavy, &nch));
  }
  PRGB_TRY(build_inv(g->outdeg, n, keep, &g->inv, s));
  return PR_OK;
}

}  // namespace prgb
