// octgrav_host_mlp.cpp -- C ABI of the learned opening criterion: the network
// handed to a tree (BF16 weights), training samples and labels from the walk,
// the gradient and the training loop (Sec. 2.2's opening test replaced by a
// network, with the plain test as fallback).
#include "octgrav_host.h"
#include "octgrav_mlp.h"

using namespace ogh;

extern "C" {

// ---- learned opening criterion

static uint16_t to_bf16(float f) {  // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return static_cast<uint16_t>(u >> 16);
  u += 0x7fffu + ((u >> 16) & 1u);
  return static_cast<uint16_t>(u >> 16);
}
static uint32_t pack2(float lo, float hi) { return to_bf16(lo) | (static_cast<uint32_t>(to_bf16(hi)) << 16); }

int octgrav_set_criterion(octgrav_tree* t, const float* record, double tau, double theta_lo, double theta_hi,
                          double theta_fb) {
  if (!t) return fail(OCTGRAV_ERR_ARG, "tree is NULL");
  if (!record) {
    if (!t->learned) return OCTGRAV_OK;
    t->learned = false;
    return ogh::rebuild_items(t);  // plain-criterion items (item_split)
  }
  if (!(theta_lo >= 0 && theta_hi >= theta_lo && theta_fb >= 0) || !std::isfinite(tau) || !std::isfinite(theta_hi))
    return fail(OCTGRAV_ERR_ARG, "need 0 <= theta_lo <= theta_hi, theta_fb >= 0 and a finite tau");
  const float* mu = record;
  const float* sg = record + 12;
  const float* xmin = record + 24;
  const float* xmax = record + 36;
  const float* w = record + 48;
  const float* W1 = w;
  const float* b1 = W1 + og::MLP_NH * og::MLP_NF;
  const float* W2 = b1 + og::MLP_NH;
  const float* b2 = W2 + og::MLP_NH * og::MLP_NH;
  const float* w3 = b2 + og::MLP_NH;
  og::MlpDevice D;
  std::memset(&D, 0, sizeof D);
  auto w1 = [&](int u, int k) { return k < og::MLP_NF ? W1[u * og::MLP_NF + k] : 0.f; };
  for (int j = 0; j < 8; ++j)
    for (int L = 0; L < 32; ++L) {  // B fragment of W1^T: rows k = 2(L%4)+{0,1}, +8; column u = 8j + L/4
      const int u = 8 * j + L / 4, k = 2 * (L % 4);
      D.w1f[j][L] = make_uint2(pack2(w1(u, k), w1(u, k + 1)), pack2(w1(u, k + 8), w1(u, k + 9)));
    }
  for (int kk = 0; kk < 4; ++kk)
    for (int j = 0; j < 8; ++j)
      for (int L = 0; L < 32; ++L) {
        const int u = 8 * j + L / 4, k = 16 * kk + 2 * (L % 4);
        const float* r = W2 + u * og::MLP_NH;
        D.w2f[kk][j][L] = make_uint2(pack2(r[k], r[k + 1]), pack2(r[k + 8], r[k + 9]));
      }
  for (int j = 0; j < og::MLP_NH; ++j) {
    D.b1[j] = b1[j];
    D.b2[j] = b2[j];
    D.w3[j] = w3[j];
  }
  for (int i = 0; i < 16; ++i) {
    const bool v = i < og::MLP_NF;
    D.mu[i] = v ? mu[i] : 0.f;
    D.isig[i] = v ? 1.f / sg[i] : 0.f;
    D.xmin[i] = v ? xmin[i] : 0.f;
    D.xmax[i] = v ? xmax[i] : 0.f;
  }
  D.b3 = w3[og::MLP_NH];
  D.tau = static_cast<float>(tau);
  int rc = t->dev->mlp.reserve(sizeof D);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpy(t->dev->mlp.p, &D, sizeof D, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaGetDevice(&t->mlp_device));
  const bool was = t->learned;
  t->learned = true;
  t->theta_lo = static_cast<float>(theta_lo);
  t->theta_hi = static_cast<float>(theta_hi);
  t->theta_fb = static_cast<float>(theta_fb);
  return was ? OCTGRAV_OK : ogh::rebuild_items(t);  // learned-criterion items (item_split)
}

// Host copy of the walk's FP32 opening test (same operations, no contraction).
static bool open_f32_host(const float4& g, const float4& b0, const float4& b1, float theta2, float* d2out) {
  const float h = g.w;
  const float gmin[3] = {b0.x, b0.y, b0.z}, gmax[3] = {b1.x, b1.y, b1.z}, c[3] = {g.x, g.y, g.z};
  float d[3];
  for (int k = 0; k < 3; ++k) {
    const float below = gmin[k] - (c[k] + h), above = (c[k] - h) - gmax[k];
    const float tt = below > above ? below : above;
    d[k] = tt > 0.f ? tt : 0.f;
  }
  const float d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
  if (d2out) *d2out = d2;
  return 4.0f * (h * h) >= theta2 * d2;
}

int octgrav_mlp_samples(octgrav_tree* t, const int64_t* groups, int64_t n_groups, double theta_walk, double eps,
                        float* features, float* labels, int64_t* pairs, int64_t cap, int64_t* n_out, void* stream) {
  if (!t || !groups || n_groups < 0 || !n_out) return fail(OCTGRAV_ERR_ARG, "bad argument");
  int rc = check_params(eps, theta_walk, 1.0);
  if (rc) return rc;
  if ((rc = host_images(t))) return rc;
  const int64_t ngr = static_cast<int64_t>(t->group_cell.size());
  const float th2 = static_cast<float>(theta_walk * theta_walk);
  std::vector<int32_t> s_item, s_cell;
  std::vector<int64_t> s_group;
  int max_count = 1;
  for (int64_t q = 0; q < n_groups; ++q) {
    const int64_t g = groups[q];
    if (g < 0 || g >= ngr) return fail(OCTGRAV_ERR_ARG, "group index %lld out of range", (long long)g);
    const int item = t->group_item[g];
    const int4 it = t->items[item];
    const float4 b0 = t->ibox[4 * item], b1 = t->ibox[4 * item + 1];
    max_count = std::max<int>(max_count, static_cast<int>(t->pcount[t->group_cell[g]]));
    std::vector<int32_t> stack;
    if (t->link[it.x].y > 0) stack.push_back(it.x);
    while (!stack.empty()) {
      const int node = stack.back();
      stack.pop_back();
      const int2 lk = t->link[node];
      for (int c = lk.x; c < lk.x + lk.y; ++c) {
        float d2 = 0.f;
        const bool op = open_f32_host(t->geo[c], b0, b1, th2, &d2);
        if (t->geo[c].w > 0.f && d2 > 0.f) {
          s_item.push_back(item);
          s_cell.push_back(c);
          s_group.push_back(g);
        }
        if (op && t->link[c].y > 0) stack.push_back(c);
      }
    }
  }
  const int64_t ns = static_cast<int64_t>(s_item.size());
  *n_out = ns;
  if (!features || !labels || cap <= 0 || ns == 0) return OCTGRAV_OK;
  const int64_t nw = std::min(ns, cap);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!t->uploaded || t->sysp_dirty) {
    if ((rc = upload(t, st))) return rc;
  }
  // reference accelerations: the same walk at theta = 0.3 with the plain test
  const bool learned = t->learned;
  t->learned = false;
  if ((rc = t->dev->out.reserve(sizeof(float4) * t->n))) { t->learned = learned; return rc; }
  rc = launch(t, eps, 0.3, 1.0, static_cast<float4*>(t->dev->out.p), st);
  t->learned = learned;
  if (rc) return rc;
  if ((rc = read_status(t, st))) return rc;
  // per-cell (first, count) and FP64 moments
  const int64_t nc = t->n_cells;
  std::vector<int2> fc(nc);
  for (int64_t c = 0; c < nc; ++c) fc[c] = make_int2(t->cfirst[c], static_cast<int>(t->pcount[c]));
  DevBuf b_item, b_cell, b_fc, b_com, b_M, b_S, b_feat, b_lab;
  if ((rc = b_item.reserve(4 * nw)) || (rc = b_cell.reserve(4 * nw)) || (rc = b_fc.reserve(8 * nc)) ||
      (rc = b_com.reserve(24 * nc)) || (rc = b_M.reserve(8 * nc)) || (rc = b_S.reserve(48 * nc)) ||
      (rc = b_feat.reserve(4 * og::MLP_NF * nw)) || (rc = b_lab.reserve(8 * nw)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(b_item.p, s_item.data(), 4 * nw, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b_cell.p, s_cell.data(), 4 * nw, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b_fc.p, fc.data(), 8 * nc, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b_com.p, t->com.data(), 24 * nc, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b_M.p, t->M.data(), 8 * nc, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b_S.p, t->S.data(), 48 * nc, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(b_lab.p, 0, 8 * nw, st));
  og::MlpSampleArgs a{};
  a.n = static_cast<int>(nw);
  a.chunks = (max_count + 31) / 32;
  a.item = static_cast<const int*>(b_item.p);
  a.cell = static_cast<const int*>(b_cell.p);
  a.items = static_cast<const int4*>(t->dev->items.p);
  a.ibox = static_cast<const float4*>(t->dev->ibox.p);
  a.geo = static_cast<const float4*>(t->dev->geo.p);
  a.mp = static_cast<const float4*>(t->dev->mp.p);
  a.parts = static_cast<const float4*>(t->dev->parts.p);
  a.link_first_count = static_cast<const int2*>(b_fc.p);
  a.com64 = static_cast<const double*>(b_com.p);
  a.M64 = static_cast<const double*>(b_M.p);
  a.S64 = static_cast<const double*>(b_S.p);
  a.aref = static_cast<const float4*>(t->dev->out.p);
  a.eps2 = eps * eps;
  a.n_group = t->n_group;
  a.feat = static_cast<float*>(b_feat.p);
  a.label64 = static_cast<double*>(b_lab.p);
  cudaError_t e = og::mlp_sample_features(a, st);
  if (e == cudaSuccess) e = og::mlp_sample_labels(a, st);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "sample kernels failed: %s", cudaGetErrorString(e));
  std::vector<double> lab(nw);
  CUDA_TRY(cudaMemcpyAsync(features, b_feat.p, 4 * og::MLP_NF * nw, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(lab.data(), b_lab.p, 8 * nw, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t k = 0; k < nw; ++k) {
    labels[k] = static_cast<float>(lab[k]);
    if (pairs) {
      pairs[2 * k] = s_group[k];
      pairs[2 * k + 1] = s_cell[k];
    }
  }
  return OCTGRAV_OK;
}

static double splitmix_uniform(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return static_cast<double>(z >> 11) * (1.0 / 9007199254740992.0);
}

int octgrav_mlp_grad(const float* params, const float* x, const float* target, int64_t n, float* grad, float* loss,
                     void* stream) {
  if (!params || !x || !target || n < 1 || n > (1 << 30) || !grad) return fail(OCTGRAV_ERR_ARG, "bad argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevBuf bw, bx, bt, bg, bl;
  int rc;
  if ((rc = bw.reserve(4 * og::MLP_NPARAM)) || (rc = bx.reserve(4 * og::MLP_NF * n)) || (rc = bt.reserve(4 * n)) ||
      (rc = bg.reserve(4 * og::MLP_NPARAM)) || (rc = bl.reserve(4)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(bw.p, params, 4 * og::MLP_NPARAM, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(bx.p, x, 4 * og::MLP_NF * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(bt.p, target, 4 * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(bg.p, 0, 4 * og::MLP_NPARAM, st));
  CUDA_TRY(cudaMemsetAsync(bl.p, 0, 4, st));
  cudaError_t e = og::mlp_grad(static_cast<float*>(bw.p), static_cast<float*>(bx.p), static_cast<float*>(bt.p),
                               static_cast<int>(n), static_cast<int>(n), 0, 0, true, static_cast<float*>(bg.p),
                               static_cast<float*>(bl.p), st);
  if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "gradient kernel failed: %s", cudaGetErrorString(e));
  CUDA_TRY(cudaMemcpyAsync(grad, bg.p, 4 * og::MLP_NPARAM, cudaMemcpyDeviceToHost, st));
  float l = 0;
  CUDA_TRY(cudaMemcpyAsync(&l, bl.p, 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  return OCTGRAV_OK;
}

int octgrav_mlp_train(const float* features, const float* labels, int64_t n, int steps, int batch, double lr,
                      uint64_t seed, float* record, float* final_loss, void* stream) {
  if (!features || !labels || !record || n < 2 || n > (1 << 30) || steps < 1 || batch < 1 || !(lr > 0))
    return fail(OCTGRAV_ERR_ARG, "bad argument");
  const int F = og::MLP_NF;
  // targets: log10 of the error label; inputs standardised per feature
  std::vector<float> y(n), X(static_cast<size_t>(n) * F);
  double mu[og::MLP_NF] = {0}, sd[og::MLP_NF] = {0};
  for (int64_t k = 0; k < n; ++k)
    for (int i = 0; i < F; ++i) mu[i] += features[k * F + i];
  for (int i = 0; i < F; ++i) mu[i] /= static_cast<double>(n);
  for (int64_t k = 0; k < n; ++k)
    for (int i = 0; i < F; ++i) sd[i] += (features[k * F + i] - mu[i]) * (features[k * F + i] - mu[i]);
  for (int i = 0; i < F; ++i) sd[i] = std::max(std::sqrt(sd[i] / static_cast<double>(n)), 1e-6);
  float xmin[og::MLP_NF], xmax[og::MLP_NF];
  for (int i = 0; i < F; ++i) { xmin[i] = INFINITY; xmax[i] = -INFINITY; }
  for (int64_t k = 0; k < n; ++k) {
    y[k] = static_cast<float>(std::log10(std::max(static_cast<double>(labels[k]), 1e-12)));
    for (int i = 0; i < F; ++i) {
      const float v = static_cast<float>((features[k * F + i] - mu[i]) / sd[i]);
      X[k * F + i] = v;
      xmin[i] = std::min(xmin[i], v);
      xmax[i] = std::max(xmax[i], v);
    }
  }
  // He-uniform initialisation from a counter-based generator
  std::vector<float> w(og::MLP_NPARAM, 0.f);
  uint64_t rs = seed;
  const int NH = og::MLP_NH;
  for (int k = 0; k < NH * F; ++k) w[k] = static_cast<float>((2 * splitmix_uniform(rs) - 1) * std::sqrt(6.0 / F));
  float* W2 = w.data() + NH * F + NH;
  for (int k = 0; k < NH * NH; ++k) W2[k] = static_cast<float>((2 * splitmix_uniform(rs) - 1) * std::sqrt(6.0 / NH));
  float* w3 = W2 + NH * NH + NH;
  for (int k = 0; k < NH; ++k) w3[k] = static_cast<float>((2 * splitmix_uniform(rs) - 1) * std::sqrt(3.0 / NH));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevBuf bx, by, bw, bm, bv, bg, bl;
  int rc;
  if ((rc = bx.reserve(4 * X.size())) || (rc = by.reserve(4 * n)) || (rc = bw.reserve(4 * og::MLP_NPARAM)) ||
      (rc = bm.reserve(4 * og::MLP_NPARAM)) || (rc = bv.reserve(4 * og::MLP_NPARAM)) ||
      (rc = bg.reserve(4 * og::MLP_NPARAM)) || (rc = bl.reserve(4)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(bx.p, X.data(), 4 * X.size(), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(by.p, y.data(), 4 * n, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(bw.p, w.data(), 4 * og::MLP_NPARAM, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(bm.p, 0, 4 * og::MLP_NPARAM, st));
  CUDA_TRY(cudaMemsetAsync(bv.p, 0, 4 * og::MLP_NPARAM, st));
  const int B = static_cast<int>(std::min<int64_t>(batch, n));
  for (int k = 1; k <= steps; ++k) {
    CUDA_TRY(cudaMemsetAsync(bg.p, 0, 4 * og::MLP_NPARAM, st));
    CUDA_TRY(cudaMemsetAsync(bl.p, 0, 4, st));
    cudaError_t e = og::mlp_grad(static_cast<float*>(bw.p), static_cast<float*>(bx.p), static_cast<float*>(by.p),
                                 static_cast<int>(n), B, k, seed, false, static_cast<float*>(bg.p),
                                 static_cast<float*>(bl.p), st);
    if (e == cudaSuccess)
      e = og::mlp_adam(static_cast<float*>(bw.p), static_cast<float*>(bm.p), static_cast<float*>(bv.p),
                       static_cast<float*>(bg.p), static_cast<float>(lr), k, st);
    if (e != cudaSuccess) return fail(OCTGRAV_ERR_CUDA, "training kernels failed: %s", cudaGetErrorString(e));
  }
  float l = 0;
  CUDA_TRY(cudaMemcpyAsync(w.data(), bw.p, 4 * og::MLP_NPARAM, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(&l, bl.p, 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  // The range limits are the training extremes widened by kRangeMargin standard
  // deviations: an input equal to an extreme is in range however it is
  // rounded (several inputs take discrete values -- counts, cell sizes -- that
  // sit exactly on an extreme, and an FP32 and an FP64 evaluation of them
  // differ in the last bits).
  constexpr float kRangeMargin = 1e-3f;
  for (int i = 0; i < F; ++i) {
    record[i] = static_cast<float>(mu[i]);
    record[12 + i] = static_cast<float>(sd[i]);
    record[24 + i] = xmin[i] - kRangeMargin;
    record[36 + i] = xmax[i] + kRangeMargin;
  }
  std::memcpy(record + 48, w.data(), 4 * og::MLP_NPARAM);
  if (final_loss) *final_loss = l;
  return OCTGRAV_OK;
}

}  // extern "C"
