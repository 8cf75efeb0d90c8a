// Lens maps into host memory (Sec. 2.1 maps, the A5 outputs), with the device-to-host copies
// overlapped with the computation: the grid is split into bands of whole rows; band k is
// computed on the caller's stream into one of two device slots of the caller's workspace
// while the band before it is copied to the host on a second (library) stream.  With the
// maps of a 4096^2 grid (604 MB) the copy over the host link takes longer than the
// computation, so the call then costs about the copy time plus one band's computation.
#include <mutex>

namespace lf {

// Device bytes of one band slot (each map 256-byte aligned): ax, ay, mu (FP64) and kappa,
// g1, g2 (FP32) for `px` pixels.
static size_t hostio_slot_bytes(long long px) {
  auto up = [](size_t b) { return (b + 255u) & ~(size_t)255u; };
  return 3 * up((size_t)px * 8u) + 3 * up((size_t)px * 4u);
}

// Rows per band for `bands` requested bands of an ny-row grid: a multiple of the mixed maps'
// 16-row anchor tiles, so that every band's tiles (and anchors) are those of the whole grid.
static int hostio_rows(int ny, int bands) {
  const int nb = std::min(bands, ny);
  const int rows = (ny + nb - 1) / nb;
  return std::min(ny, (rows + 15) / 16 * 16);
}

// One non-blocking copy stream per device, created on first use and kept for the process.
static cudaStream_t hostio_copy_stream(int dev, lf_status& st) {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  st = LF_OK;
  if (dev < 0 || dev >= 64) { st = fail(LF_EUNSUPPORTED, "device index %d beyond 63", dev); return nullptr; }
  std::lock_guard<std::mutex> lock(mu);
  if (!streams[dev]) {
    cudaError_t e = cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    if (e != cudaSuccess) { st = fail(LF_ECUDA, "cudaStreamCreateWithFlags: %s", cudaGetErrorString(e)); return nullptr; }
  }
  return streams[dev];
}

}  // namespace lf

using namespace lf;

extern "C" size_t lf_jacobian_grid_host_workspace(const lf_grid* grid, int32_t bands) {
  if (!grid || grid->nx <= 0 || grid->ny <= 0 || bands < 1) return 0;
  const long long px = (long long)grid->nx * hostio_rows(grid->ny, bands);
  return 2 * hostio_slot_bytes(px);
}

extern "C" lf_status lf_jacobian_grid_host(const lf_plane* plane, const lf_grid* grid, double a_dis,
                                           int32_t precision, double* ax, double* ay, float* kappa,
                                           float* g1, float* g2, double* mu, int32_t bands,
                                           void* workspace, size_t workspace_bytes, void* stream) {
  LF_TRY(check_grid(grid));
  LF_TRY(check_plane(plane));
  if (!(a_dis > 0.0 && a_dis <= 1.0)) return fail(LF_EINVAL, "a_dis must be in (0, 1]");
  if (precision < LF_FP64 || precision > LF_FF) return fail(LF_EINVAL, "unknown precision");
  if (bands < 1) return fail(LF_EINVAL, "bands must be >= 1");
  const size_t need = lf_jacobian_grid_host_workspace(grid, bands);
  if (!workspace || workspace_bytes < need)
    return fail(LF_EINVAL, "workspace must hold %zu bytes (lf_jacobian_grid_host_workspace)", need);
  if (((uintptr_t)workspace) & 255u) return fail(LF_EINVAL, "workspace must be 256-byte aligned");
  if (!(ax || ay || kappa || g1 || g2 || mu)) return LF_OK;

  const int nx = grid->nx, ny = grid->ny, rows = hostio_rows(ny, bands);
  const int nb = (ny + rows - 1) / rows;
  const long long slot_px = (long long)nx * rows;
  int dev = 0;
  LF_CUDA(cudaGetDevice(&dev));
  lf_status st = LF_OK;
  cudaStream_t cs = hostio_copy_stream(dev, st);
  if (st != LF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;

  // the two device slots
  struct Slot { double *ax, *ay, *mu; float *kappa, *g1, *g2; } slot[2];
  for (int q = 0; q < 2; ++q) {
    unsigned char* b = (unsigned char*)workspace + (size_t)q * hostio_slot_bytes(slot_px);
    const size_t d = ((size_t)slot_px * 8u + 255u) & ~(size_t)255u, f = ((size_t)slot_px * 4u + 255u) & ~(size_t)255u;
    slot[q].ax = (double*)b; slot[q].ay = (double*)(b + d); slot[q].mu = (double*)(b + 2 * d);
    slot[q].kappa = (float*)(b + 3 * d); slot[q].g1 = (float*)(b + 3 * d + f); slot[q].g2 = (float*)(b + 3 * d + 2 * f);
  }
  cudaEvent_t computed[2] = {}, copied[2] = {}, fin = nullptr;
  auto destroy = [&]() {
    for (int q = 0; q < 2; ++q) {
      if (computed[q]) cudaEventDestroy(computed[q]);
      if (copied[q]) cudaEventDestroy(copied[q]);
    }
    if (fin) cudaEventDestroy(fin);
  };
  for (int q = 0; q < 2 && st == LF_OK; ++q) {
    if (cudaEventCreateWithFlags(&computed[q], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&copied[q], cudaEventDisableTiming) != cudaSuccess)
      st = fail(LF_ECUDA, "cudaEventCreateWithFlags failed");
  }
  if (st == LF_OK && cudaEventCreateWithFlags(&fin, cudaEventDisableTiming) != cudaSuccess)
    st = fail(LF_ECUDA, "cudaEventCreateWithFlags failed");
  if (st != LF_OK) { destroy(); return st; }

  cudaError_t ce = cudaSuccess;
  for (int k = 0; k < nb && st == LF_OK && ce == cudaSuccess; ++k) {
    const int q = k & 1, r0 = k * rows, nr = std::min(rows, ny - r0);
    const Slot& sl = slot[q];
    // the slot is free once the copies of the band two before this one are done
    if (k >= 2) ce = cudaStreamWaitEvent(s, copied[q], 0);
    if (ce != cudaSuccess) break;
    lf_grid gb = *grid;
    gb.y0 = grid->y0 + (double)r0 * grid->dy;
    gb.ny = nr;
    st = lf_jacobian_grid(plane, &gb, a_dis, precision, ax ? sl.ax : nullptr, ay ? sl.ay : nullptr,
                          kappa ? sl.kappa : nullptr, g1 ? sl.g1 : nullptr, g2 ? sl.g2 : nullptr,
                          mu ? sl.mu : nullptr, s);
    if (st != LF_OK) break;
    if ((ce = cudaEventRecord(computed[q], s)) != cudaSuccess) break;
    if ((ce = cudaStreamWaitEvent(cs, computed[q], 0)) != cudaSuccess) break;
    const size_t off = (size_t)r0 * nx, n = (size_t)nr * nx;
    if (ax && ce == cudaSuccess) ce = cudaMemcpyAsync(ax + off, sl.ax, n * 8u, cudaMemcpyDeviceToHost, cs);
    if (ay && ce == cudaSuccess) ce = cudaMemcpyAsync(ay + off, sl.ay, n * 8u, cudaMemcpyDeviceToHost, cs);
    if (mu && ce == cudaSuccess) ce = cudaMemcpyAsync(mu + off, sl.mu, n * 8u, cudaMemcpyDeviceToHost, cs);
    if (kappa && ce == cudaSuccess) ce = cudaMemcpyAsync(kappa + off, sl.kappa, n * 4u, cudaMemcpyDeviceToHost, cs);
    if (g1 && ce == cudaSuccess) ce = cudaMemcpyAsync(g1 + off, sl.g1, n * 4u, cudaMemcpyDeviceToHost, cs);
    if (g2 && ce == cudaSuccess) ce = cudaMemcpyAsync(g2 + off, sl.g2, n * 4u, cudaMemcpyDeviceToHost, cs);
    if (ce == cudaSuccess) ce = cudaEventRecord(copied[q], cs);
  }
  // the caller's stream is ordered after every copy issued, also when a step above failed
  cudaError_t ce2 = cudaEventRecord(fin, cs);
  if (ce2 == cudaSuccess) ce2 = cudaStreamWaitEvent(s, fin, 0);
  destroy();
  if (st != LF_OK) return st;
  if (ce != cudaSuccess) return fail(LF_ECUDA, "%s", cudaGetErrorString(ce));
  if (ce2 != cudaSuccess) return fail(LF_ECUDA, "%s", cudaGetErrorString(ce2));
  return LF_OK;
}
