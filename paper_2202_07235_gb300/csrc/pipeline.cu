// Host-input alignment pipeline: images and templates in (pinned) host memory,
// best/arg (and log-sum-exp) back to host memory, with the host-to-device
// copies of one chunk of images overlapping the compression and alignment of
// the previous chunk. Only the half ring psi < pi of each polar sample array is
// copied: the compression reads no other samples (real images,
// A(k, psi + pi) = conj A(k, psi)).
//
// Streams: `stream` runs compression and alignment, `copy_stream` every copy.
// Chunk c uses polar buffer c mod 2 and output buffer c mod 2; events order
//   H2D(c) -> compress(c)          (input ready)
//   compress(c) -> H2D(c + 2)      (polar buffer free)
//   align(c) -> D2H(c)             (results ready)
//   D2H(c) -> align(c + 2)         (output buffer free).
// On the copy stream H2D(c + 1) is enqueued before D2H(c), so it runs while
// chunk c is aligned. At return, `stream` waits for the last copy, so
// synchronising `stream` makes every result visible on the host.
#include "operand.cuh"

namespace {

constexpr size_t kAlign = 256;
inline size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct PipeLayout {
  size_t polar, tpolar, cA, cB, best, arg, lse, total;
};

PipeLayout pipe_layout(int R, int Q, int H, int T, int N_B, int chunk, int precision, bool want_lse) {
  PipeLayout L{};
  const size_t ring = (size_t)R * Q * sizeof(float2);
  L.polar = up((size_t)chunk * ring);
  L.tpolar = up((size_t)N_B * ring);
  L.cA = up(rsvd_compressed_bytes(chunk, T, H, Q, precision));
  L.cB = up(rsvd_compressed_bytes(N_B, 1, H, Q, precision));
  const size_t outs = (size_t)chunk * N_B;
  L.best = up(outs * sizeof(float));
  L.arg = up(outs * sizeof(int32_t));
  L.lse = want_lse ? up(outs * sizeof(float)) : 0;
  L.total = 2 * L.polar + L.tpolar + L.cA + L.cB + 2 * (L.best + L.arg + L.lse);
  return L;
}

struct Events {
  cudaEvent_t ev[8] = {};
  int n = 0;
  bool make() {
    for (n = 0; n < 8; ++n)
      if (cudaEventCreateWithFlags(&ev[n], cudaEventDisableTiming) != cudaSuccess) return false;
    return true;
  }
  ~Events() {
    for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
  }
};

}  // namespace

extern "C" size_t rsvd_align_host_workspace_bytes(int R, int Q, int H, int T, int N_B, int chunk, int precision,
                                                  int want_lse) {
  if (R <= 0 || Q <= 0 || H <= 0 || T <= 0 || N_B <= 0 || chunk <= 0) return 0;
  if (rsvd_compressed_bytes(chunk, T, H, Q, precision) == 0) return 0;
  return pipe_layout(R, Q, H, T, N_B, chunk, precision, want_lse != 0).total;
}

extern "C" int rsvd_align_best_host(int R, int Q, const double* k, const double* w, const double* U, int H,
                                    const void* images, int N_A, const double* deltas, int T,
                                    const void* templates, int N_B, int precision, float inv_sigma2,
                                    float* best, int32_t* arg, float* lse, int chunk, void* workspace,
                                    size_t workspace_bytes, void* stream, void* copy_stream) {
  if (!k || !w || !U || !images || !templates || !best || !arg || R <= 0 || Q <= 0 || H <= 0 || N_A <= 0 ||
      N_B <= 0 || T <= 0 || chunk <= 0 || (T > 1 && !deltas))
    return RSVD_EINVAL;
  if (Q % 2) return RSVD_EUNSUPPORTED;
  if (stream == copy_stream) return RSVD_EINVAL;  // the overlap needs two streams
  chunk = chunk < N_A ? chunk : N_A;
  const bool want_lse = lse != nullptr;
  const size_t need = rsvd_align_host_workspace_bytes(R, Q, H, T, N_B, chunk, precision, want_lse ? 1 : 0);
  if (need == 0) return RSVD_EUNSUPPORTED;
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & (kAlign - 1))) return RSVD_EWORKSPACE;
  const PipeLayout L = pipe_layout(R, Q, H, T, N_B, chunk, precision, want_lse);
  char* ws = static_cast<char*>(workspace);
  char* polar[2] = {ws, ws + L.polar};
  char* tpolar = ws + 2 * L.polar;
  char* cA = tpolar + L.tpolar;
  char* cB = cA + L.cA;
  char* outb = cB + L.cB;
  float* best_d[2];
  int32_t* arg_d[2];
  float* lse_d[2];
  for (int b = 0; b < 2; ++b) {
    char* o = outb + b * (L.best + L.arg + L.lse);
    best_d[b] = reinterpret_cast<float*>(o);
    arg_d[b] = reinterpret_cast<int32_t*>(o + L.best);
    lse_d[b] = want_lse ? reinterpret_cast<float*>(o + L.best + L.arg) : nullptr;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream), cp = static_cast<cudaStream_t>(copy_stream);
  Events E;
  if (!E.make()) return RSVD_ECUDA;
  cudaEvent_t ev_in[2] = {E.ev[0], E.ev[1]}, ev_used[2] = {E.ev[2], E.ev[3]};
  cudaEvent_t ev_done[2] = {E.ev[4], E.ev[5]}, ev_back[2] = {E.ev[6], E.ev[7]};
  const size_t pitch = (size_t)Q * sizeof(float2), half = pitch / 2;
  auto h2d = [&](void* dst, const void* src, size_t rings) {  // psi < pi of each ring
    return cudaMemcpy2DAsync(dst, pitch, src, pitch, half, rings, cudaMemcpyHostToDevice, cp) == cudaSuccess;
  };
  // The first chunk is a quarter of the others: the first alignment waits for
  // the templates and the whole first chunk to arrive, and a smaller first
  // chunk shortens that fill; the later copies hide behind the kernels.
  const int first = chunk >= 8 ? chunk / 4 : chunk;
  const int nchunk = 1 + (N_A - first + chunk - 1) / chunk;
  auto start = [&](int c) { return c == 0 ? 0 : first + (c - 1) * chunk; };
  auto count = [&](int c) { return c == 0 ? min(first, N_A) : min(chunk, N_A - start(c)); };
  // templates: copy (copy stream), compress (compute stream)
  if (!h2d(tpolar, templates, (size_t)N_B * R)) return RSVD_ECUDA;
  if (cudaEventRecord(ev_back[1], cp) != cudaSuccess || cudaStreamWaitEvent(st, ev_back[1], 0) != cudaSuccess)
    return RSVD_ECUDA;
  int rc = rsvd_compress(R, Q, k, w, U, H, tpolar, N_B, nullptr, 1, precision, cB, stream);
  if (rc != RSVD_OK) return rc;
  auto copy_in = [&](int c) -> int {
    const int b = c & 1, n0 = start(c), n = count(c);
    if (c >= 2 && cudaStreamWaitEvent(cp, ev_used[b], 0) != cudaSuccess) return RSVD_ECUDA;
    if (!h2d(polar[b], static_cast<const char*>(images) + (size_t)n0 * R * pitch, (size_t)n * R)) return RSVD_ECUDA;
    return cudaEventRecord(ev_in[b], cp) == cudaSuccess ? RSVD_OK : RSVD_ECUDA;
  };
  if ((rc = copy_in(0)) != RSVD_OK) return rc;
  for (int c = 0; c < nchunk; ++c) {
    const int b = c & 1, n0 = start(c), n = count(c);
    if (c + 1 < nchunk && (rc = copy_in(c + 1)) != RSVD_OK) return rc;  // overlaps chunk c's work
    if (cudaStreamWaitEvent(st, ev_in[b], 0) != cudaSuccess) return RSVD_ECUDA;
    rc = rsvd_compress(R, Q, k, w, U, H, polar[b], n, deltas, T, precision, cA, stream);
    if (rc != RSVD_OK) return rc;
    if (cudaEventRecord(ev_used[b], st) != cudaSuccess) return RSVD_ECUDA;
    if (c >= 2 && cudaStreamWaitEvent(st, ev_back[b], 0) != cudaSuccess) return RSVD_ECUDA;
    rc = rsvd_align_best(cA, n, T, cB, N_B, H, Q, precision, inv_sigma2, best_d[b], arg_d[b], lse_d[b], stream);
    if (rc != RSVD_OK) return rc;
    if (cudaEventRecord(ev_done[b], st) != cudaSuccess || cudaStreamWaitEvent(cp, ev_done[b], 0) != cudaSuccess)
      return RSVD_ECUDA;
    const size_t outs = (size_t)n * N_B, o = (size_t)n0 * N_B;
    if (cudaMemcpyAsync(best + o, best_d[b], outs * sizeof(float), cudaMemcpyDeviceToHost, cp) != cudaSuccess ||
        cudaMemcpyAsync(arg + o, arg_d[b], outs * sizeof(int32_t), cudaMemcpyDeviceToHost, cp) != cudaSuccess)
      return RSVD_ECUDA;
    if (want_lse &&
        cudaMemcpyAsync(lse + o, lse_d[b], outs * sizeof(float), cudaMemcpyDeviceToHost, cp) != cudaSuccess)
      return RSVD_ECUDA;
    if (cudaEventRecord(ev_back[b], cp) != cudaSuccess) return RSVD_ECUDA;
  }
  // the caller's stream waits for the last copies back
  if (cudaStreamWaitEvent(st, ev_back[(nchunk - 1) & 1], 0) != cudaSuccess) return RSVD_ECUDA;
  return RSVD_OK;
}

// ---------------------------------------------------------------------------
// Per-CTF-group alignment (section 3.5): the images of group g (rows
// offsets[g] .. offsets[g+1]-1) against the templates compressed with the
// group's target vectors, each group compressed and aligned on one of the
// caller's streams (round robin), so that consecutive groups' kernels overlap
// instead of each launch ending in a partly filled wave.
// ---------------------------------------------------------------------------
namespace {

struct GroupLayout {
  size_t cA, cB, per_stream;
};

GroupLayout group_layout(int Q, int H, int T, int N_B, int max_group, int precision) {
  GroupLayout L{};
  L.cA = up(rsvd_compressed_bytes(max_group, T, H, Q, precision));
  L.cB = up(rsvd_compressed_bytes(N_B, 1, H, Q, precision));
  L.per_stream = L.cA + L.cB;
  return L;
}

}  // namespace

extern "C" size_t rsvd_align_grouped_workspace_bytes(int Q, int H, int T, int N_B, int max_group, int precision,
                                                     int n_streams) {
  if (Q <= 0 || H <= 0 || T <= 0 || N_B <= 0 || max_group <= 0 || n_streams <= 0) return 0;
  if (rsvd_compressed_bytes(max_group, T, H, Q, precision) == 0) return 0;
  return group_layout(Q, H, T, N_B, max_group, precision).per_stream * (size_t)n_streams;
}

extern "C" int rsvd_align_grouped(int R, int Q, const double* k, const double* w, const double* U,
                                  const double* U_targets, int H, const void* images, const int* offsets, int G,
                                  const double* deltas, int T, const void* templates, int N_B, int precision,
                                  float* best, int32_t* arg, void* workspace, size_t workspace_bytes,
                                  void* const* streams, int n_streams) {
  if (!k || !w || !U || !U_targets || !images || !offsets || !templates || !best || !arg || !streams || R <= 0 ||
      Q <= 0 || H <= 0 || G <= 0 || T <= 0 || N_B <= 0 || n_streams <= 0 || (T > 1 && !deltas))
    return RSVD_EINVAL;
  int max_group = 0;
  for (int g = 0; g < G; ++g) {
    if (offsets[g + 1] < offsets[g] || offsets[g] < 0) return RSVD_EINVAL;
    max_group = max(max_group, offsets[g + 1] - offsets[g]);
  }
  if (max_group == 0) return RSVD_OK;
  for (int i = 0; i < n_streams; ++i)
    for (int j = 0; j < i; ++j)
      if (streams[i] == streams[j]) return RSVD_EINVAL;
  const size_t need = rsvd_align_grouped_workspace_bytes(Q, H, T, N_B, max_group, precision, n_streams);
  if (need == 0) return RSVD_EUNSUPPORTED;
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & (kAlign - 1))) return RSVD_EWORKSPACE;
  const GroupLayout L = group_layout(Q, H, T, N_B, max_group, precision);
  cudaStream_t s0 = static_cast<cudaStream_t>(streams[0]);
  cudaEvent_t ev[64];
  const int ns = n_streams < 64 ? n_streams : 64;
  int made = 0;
  auto cleanup = [&]() {
    for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  };
  for (; made < ns; ++made)
    if (cudaEventCreateWithFlags(&ev[made], cudaEventDisableTiming) != cudaSuccess) {
      cleanup();
      return RSVD_ECUDA;
    }
  // fork: every stream starts after the work already queued on the first
  int rc = RSVD_OK;
  if (cudaEventRecord(ev[0], s0) != cudaSuccess) rc = RSVD_ECUDA;
  for (int i = 1; i < ns && rc == RSVD_OK; ++i)
    if (cudaStreamWaitEvent(static_cast<cudaStream_t>(streams[i]), ev[0], 0) != cudaSuccess) rc = RSVD_ECUDA;
  const size_t ring = (size_t)R * Q * sizeof(float2);
  const size_t uH = (size_t)R * H;
  for (int g = 0; g < G && rc == RSVD_OK; ++g) {
    const int a0 = offsets[g], n = offsets[g + 1] - a0;
    if (n == 0) continue;
    const int si = g % ns;
    void* st = streams[si];
    char* cA = static_cast<char*>(workspace) + (size_t)si * L.per_stream;
    char* cB = cA + L.cA;
    rc = rsvd_compress(R, Q, k, w, U + g * uH, H, static_cast<const char*>(images) + (size_t)a0 * ring, n, deltas, T,
                       precision, cA, st);
    if (rc == RSVD_OK) rc = rsvd_compress(R, Q, k, w, U_targets + g * uH, H, templates, N_B, nullptr, 1, precision, cB, st);
    if (rc == RSVD_OK)
      rc = rsvd_align_best(cA, n, T, cB, N_B, H, Q, precision, 1.0f, best + (size_t)a0 * N_B, arg + (size_t)a0 * N_B,
                           nullptr, st);
  }
  // join: the first stream waits for all the others
  for (int i = 1; i < ns; ++i) {
    if (cudaEventRecord(ev[i], static_cast<cudaStream_t>(streams[i])) != cudaSuccess ||
        cudaStreamWaitEvent(s0, ev[i], 0) != cudaSuccess)
      if (rc == RSVD_OK) rc = RSVD_ECUDA;
  }
  cleanup();
  return rc;
}

// ---------------------------------------------------------------------------
// Host-input volume alignment (section 4): volumes and targets in (pinned) host
// memory, best/arg back to host memory; the copy of chunk c + 1 of the volumes
// overlaps the compression and alignment of chunk c, with the same buffers and
// events as the image pipeline above.
// ---------------------------------------------------------------------------
namespace {

struct VolPipeLayout {
  size_t vol, tgt, cA, cB, best, arg, total;
};

VolPipeLayout vol_pipe_layout(int R, int L, int HC, int N_B, int chunk) {
  VolPipeLayout P{};
  const size_t lm = (size_t)(L + 1) * (2 * L + 1) * sizeof(float2);
  P.vol = up((size_t)chunk * R * lm);
  P.tgt = up((size_t)N_B * R * lm);
  P.cA = up((size_t)chunk * HC * lm);
  P.cB = up((size_t)N_B * HC * lm);
  const size_t outs = (size_t)chunk * N_B;
  P.best = up(outs * sizeof(float));
  P.arg = up(outs * sizeof(int32_t));
  P.total = 2 * P.vol + P.tgt + P.cA + P.cB + 2 * (P.best + P.arg);
  return P;
}

}  // namespace

extern "C" size_t rsvd_align_volumes_host_workspace_bytes(int R, int L, int HC, int N_B, int chunk) {
  if (R <= 0 || L < 1 || HC <= 0 || N_B <= 0 || chunk <= 0) return 0;
  return vol_pipe_layout(R, L, HC, N_B, chunk).total;
}

extern "C" int rsvd_align_volumes_host(int R, int L, const double* w, const double* U, int HC, const double* V, int HD,
                                       const float* tables, int n_beta, int Mp, const void* volumes, int N_A,
                                       const void* targets, int N_B, int real_volumes, float* best, int32_t* arg,
                                       int chunk, void* workspace, size_t workspace_bytes, void* stream,
                                       void* copy_stream) {
  if (!w || !U || !V || !tables || !volumes || !targets || !best || !arg || R <= 0 || L < 1 || HC <= 0 || HD <= 0 ||
      n_beta <= 0 || N_A <= 0 || N_B <= 0 || chunk <= 0)
    return RSVD_EINVAL;
  if (stream == copy_stream) return RSVD_EINVAL;
  chunk = chunk < N_A ? chunk : N_A;
  const size_t need = rsvd_align_volumes_host_workspace_bytes(R, L, HC, N_B, chunk);
  if (need == 0) return RSVD_EUNSUPPORTED;
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & (kAlign - 1))) return RSVD_EWORKSPACE;
  const VolPipeLayout P = vol_pipe_layout(R, L, HC, N_B, chunk);
  char* ws = static_cast<char*>(workspace);
  char* vol[2] = {ws, ws + P.vol};
  char* tgt = ws + 2 * P.vol;
  char* cA = tgt + P.tgt;
  char* cB = cA + P.cA;
  char* outb = cB + P.cB;
  float* best_d[2];
  int32_t* arg_d[2];
  for (int b = 0; b < 2; ++b) {
    best_d[b] = reinterpret_cast<float*>(outb + b * (P.best + P.arg));
    arg_d[b] = reinterpret_cast<int32_t*>(outb + b * (P.best + P.arg) + P.best);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream), cp = static_cast<cudaStream_t>(copy_stream);
  Events E;
  if (!E.make()) return RSVD_ECUDA;
  cudaEvent_t ev_in[2] = {E.ev[0], E.ev[1]}, ev_used[2] = {E.ev[2], E.ev[3]};
  cudaEvent_t ev_done[2] = {E.ev[4], E.ev[5]}, ev_back[2] = {E.ev[6], E.ev[7]};
  const size_t per = (size_t)R * (L + 1) * (2 * L + 1) * sizeof(float2);  // one volume
  if (cudaMemcpyAsync(tgt, targets, (size_t)N_B * per, cudaMemcpyHostToDevice, cp) != cudaSuccess ||
      cudaEventRecord(ev_back[1], cp) != cudaSuccess || cudaStreamWaitEvent(st, ev_back[1], 0) != cudaSuccess)
    return RSVD_ECUDA;
  int rc = rsvd_compress_volume(R, L, w, U, HC, tgt, N_B, cB, stream);
  if (rc != RSVD_OK) return rc;
  const int nchunk = (N_A + chunk - 1) / chunk;
  auto copy_in = [&](int c) -> int {
    const int b = c & 1, n0 = c * chunk, n = min(chunk, N_A - n0);
    if (c >= 2 && cudaStreamWaitEvent(cp, ev_used[b], 0) != cudaSuccess) return RSVD_ECUDA;
    if (cudaMemcpyAsync(vol[b], static_cast<const char*>(volumes) + (size_t)n0 * per, (size_t)n * per,
                        cudaMemcpyHostToDevice, cp) != cudaSuccess)
      return RSVD_ECUDA;
    return cudaEventRecord(ev_in[b], cp) == cudaSuccess ? RSVD_OK : RSVD_ECUDA;
  };
  if ((rc = copy_in(0)) != RSVD_OK) return rc;
  for (int c = 0; c < nchunk; ++c) {
    const int b = c & 1, n0 = c * chunk, n = min(chunk, N_A - n0);
    if (c + 1 < nchunk && (rc = copy_in(c + 1)) != RSVD_OK) return rc;
    if (cudaStreamWaitEvent(st, ev_in[b], 0) != cudaSuccess) return RSVD_ECUDA;
    if ((rc = rsvd_compress_volume(R, L, w, U, HC, vol[b], n, cA, stream)) != RSVD_OK) return rc;
    if (cudaEventRecord(ev_used[b], st) != cudaSuccess) return RSVD_ECUDA;
    if (c >= 2 && cudaStreamWaitEvent(st, ev_back[b], 0) != cudaSuccess) return RSVD_ECUDA;
    rc = (real_volumes ? rsvd_align_volumes_real : rsvd_align_volumes)(cA, n, cB, N_B, HC, L, V, HD, tables, n_beta,
                                                                        Mp, best_d[b], arg_d[b], stream);
    if (rc != RSVD_OK) return rc;
    if (cudaEventRecord(ev_done[b], st) != cudaSuccess || cudaStreamWaitEvent(cp, ev_done[b], 0) != cudaSuccess)
      return RSVD_ECUDA;
    const size_t outs = (size_t)n * N_B, o = (size_t)n0 * N_B;
    if (cudaMemcpyAsync(best + o, best_d[b], outs * sizeof(float), cudaMemcpyDeviceToHost, cp) != cudaSuccess ||
        cudaMemcpyAsync(arg + o, arg_d[b], outs * sizeof(int32_t), cudaMemcpyDeviceToHost, cp) != cudaSuccess ||
        cudaEventRecord(ev_back[b], cp) != cudaSuccess)
      return RSVD_ECUDA;
  }
  if (cudaStreamWaitEvent(st, ev_back[(nchunk - 1) & 1], 0) != cudaSuccess) return RSVD_ECUDA;
  return RSVD_OK;
}
