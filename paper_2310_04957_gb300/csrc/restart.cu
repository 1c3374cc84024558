// restart.cu -- pic_save / pic_load: the complete state of one discharge in
// one binary file, so that a run continues bit for bit after a restart.
//
// Layout: an 8-byte magic, the format version, the sizes of the two structs
// written raw (pic_config, BinMeta), the configuration with its arrays, the
// host step counter, then the device state as blobs, each prefixed by its
// byte count and checked against what the restored handle expects.  The
// particle store is written as stored (cell-relative positions, bins,
// overflow region, weight ratios of weighted handles); only the slots in use
// are written.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "handle.h"

using namespace pic;

namespace {

const char kMagic[8] = {'P', 'I', 'C', 'R', 'S', 'T', 'G', 'B'};
const uint32_t kVersion = 3;
const size_t kChunk = size_t(64) << 20;  // host bounce buffer

struct File {
  FILE *f = nullptr;
  bool ok = true;
  ~File() {
    if (f) fclose(f);
  }
  void put(const void *p, size_t n) {
    if (ok && n && fwrite(p, 1, n, f) != n) ok = false;
  }
  void get(void *p, size_t n) {
    if (ok && n && fread(p, 1, n, f) != n) ok = false;
  }
};

// A device blob: its byte count, then its bytes (through a bounded host buffer).
int put_dev(File &F, const void *d, size_t n) {
  uint64_t len = n;
  F.put(&len, sizeof(len));
  std::vector<char> buf;
  try {
    buf.resize(n < kChunk ? n : kChunk);
  } catch (const std::bad_alloc &) {
    return PIC_ENOMEM;
  }
  for (size_t off = 0; off < n && F.ok; off += kChunk) {
    const size_t m = n - off < kChunk ? n - off : kChunk;
    if (cudaMemcpy(buf.data(), static_cast<const char *>(d) + off, m, cudaMemcpyDeviceToHost) != cudaSuccess)
      return PIC_ECUDA;
    F.put(buf.data(), m);
  }
  return F.ok ? PIC_OK : PIC_EIO;
}

// Read a blob of exactly n bytes into device memory.
int get_dev(File &F, void *d, size_t n) {
  uint64_t len = 0;
  F.get(&len, sizeof(len));
  if (!F.ok || len != n) return PIC_EIO;
  std::vector<char> buf;
  try {
    buf.resize(n < kChunk ? n : kChunk);
  } catch (const std::bad_alloc &) {
    return PIC_ENOMEM;
  }
  for (size_t off = 0; off < n; off += kChunk) {
    const size_t m = n - off < kChunk ? n - off : kChunk;
    F.get(buf.data(), m);
    if (!F.ok) return PIC_EIO;
    if (cudaMemcpy(static_cast<char *>(d) + off, buf.data(), m, cudaMemcpyHostToDevice) != cudaSuccess)
      return PIC_ECUDA;
  }
  return PIC_OK;
}

// Every device array that carries state from one step to the next (or that
// pic_diag reports), with its size, in file order.  The same list serves
// saving and loading, so the two cannot drift apart.
struct Blob {
  void *p;
  size_t n;
};

std::vector<Blob> state_blobs(pic_handle *h) {
  const size_t nn = h->nn, d8 = sizeof(double), u8 = sizeof(unsigned long long);
  MgLevels tmp;
  const long long mgf = mg_plan(h->nr, h->nz, &tmp);
  std::vector<Blob> b = {
      {h->d_scalars, d8 * SC_N},
      {h->d_prop, d8 * 64},
      {h->d_pcg_out, d8 * 8},
      {h->d_ceq_out, d8 * 2},
      {h->d_counters, u8 * CNT_N},
      {h->d_flags, sizeof(uint32_t) * 2},
      {h->d_step, sizeof(uint32_t) * 2},
      {h->d_phi, d8 * nn},
      {h->d_Er, d8 * nn},
      {h->d_Ez, d8 * nn},
      {h->d_chi, d8 * nn},
      {h->d_qrhs, d8 * nn},
      {h->d_dinv, d8 * nn},
      {h->d_Gr, d8 * (size_t)(h->nz + 1) * h->nr},
      {h->d_Gz, d8 * (size_t)h->nz * (h->nr + 1)},
      {h->d_E, 2 * h->esz * nn},
      {h->d_phiL, d8 * nn},  // warm start of the next C_eq solve
      {h->mg.ws, sizeof(float) * (size_t)mgf},
      {h->mg.persist, sizeof(float) * (size_t)(h->mg.smem_floats > 0 ? h->mg.smem_floats : 1)},
      {h->mg.solves, sizeof(int)},
  };
  if (h->vahedi) {  // the Vahedi parts: phi_P (warm start) and the driven electrodes' Laplace solutions
    b.push_back({h->d_phiP, d8 * nn});
    for (int k = 0; k < h->cfg.n_drive; ++k) b.push_back({h->d_phiLd[k], d8 * nn});
  }
  for (int s = 0; s < 2; ++s) {
    b.push_back({h->d_dep[s], u8 * nn});
    b.push_back({h->d_surf[s], u8 * nn});
    b.push_back({h->d_dens_sum[s], d8 * nn});
    b.push_back({h->d_dens_avg[s], d8 * nn});
  }
  return b;
}

// Slots of a store in use: the bins, then the overflow particles.
size_t used_slots(pic_handle *h, int s, const BinMeta &m) {
  long long novf = m.ovf_n;
  if (novf > h->capacity[s] - m.ovf_base) novf = h->capacity[s] - m.ovf_base;
  if (novf < 0) novf = 0;
  return (size_t)m.ovf_base + (size_t)novf;
}

std::vector<Blob> store_columns(pic_handle *h, const Store &S, size_t used) {
  const size_t e = 4 * h->esz * used;
  std::vector<Blob> b = {{S.pa, e}, {S.pb, e}, {S.id, sizeof(unsigned long long) * used}, {S.cell, sizeof(int) * used}};
  if (h->weighted) b.push_back({S.w, h->esz * used});
  return b;
}

}  // namespace

extern "C" {

int pic_save(pic_handle *h, const char *path) {
  if (!h || !path) return PIC_EINVAL;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PIC_ECUDA;
  File F;
  F.f = fopen(path, "wb");
  if (!F.f) return PIC_EIO;
  F.put(kMagic, sizeof(kMagic));
  const uint32_t hdr[3] = {kVersion, (uint32_t)sizeof(pic_config), (uint32_t)sizeof(BinMeta)};
  F.put(hdr, sizeof(hdr));
  pic_config c = h->cfg;
  c.node_kind = nullptr;
  c.cell_kind = nullptr;
  c.cell_eps = nullptr;
  c.xs_energy = nullptr;
  c.xs_sigma = nullptr;
  F.put(&c, sizeof(c));
  F.put(h->node_kind.data(), h->node_kind.size());
  F.put(h->cell_kind.data(), h->cell_kind.size());
  F.put(h->cell_eps.data(), sizeof(double) * h->cell_eps.size());
  F.put(h->xs_E.data(), sizeof(double) * h->xs_E.size());
  F.put(h->xs_S.data(), sizeof(double) * h->xs_S.size());
  const int32_t host[2] = {(int32_t)h->step, h->started ? 1 : 0};
  F.put(host, sizeof(host));
  if (!F.ok) return PIC_EIO;
  int st;
  for (const Blob &b : state_blobs(h))
    if ((st = put_dev(F, b.p, b.n))) return st;
  for (int s = 0; s < 2; ++s) {
    const Store &S = h->st[h->cur][s];
    BinMeta m;
    if (cudaMemcpy(&m, S.meta, sizeof(m), cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
    F.put(&m, sizeof(m));
    const size_t nb = sizeof(int) * h->nbins;
    if ((st = put_dev(F, S.start, nb)) || (st = put_dev(F, S.cap, nb)) || (st = put_dev(F, S.fill, nb))) return st;
    const uint64_t used = used_slots(h, s, m);
    F.put(&used, sizeof(used));
    for (const Blob &b : store_columns(h, S, used))
      if ((st = put_dev(F, b.p, b.n))) return st;
  }
  if (!F.ok) return PIC_EIO;
  if (fflush(F.f) != 0) return PIC_EIO;
  return PIC_OK;
}

int pic_load(const char *path, void *cuda_stream, pic_handle **out) {
  if (!path || !out) return PIC_EINVAL;
  *out = nullptr;
  File F;
  F.f = fopen(path, "rb");
  if (!F.f) return PIC_EIO;
  char magic[8];
  uint32_t hdr[3];
  F.get(magic, sizeof(magic));
  F.get(hdr, sizeof(hdr));
  if (!F.ok || memcmp(magic, kMagic, sizeof(kMagic)) != 0 || hdr[0] != kVersion ||
      hdr[1] != (uint32_t)sizeof(pic_config) || hdr[2] != (uint32_t)sizeof(BinMeta))
    return PIC_EIO;
  pic_config c;
  F.get(&c, sizeof(c));
  if (!F.ok || c.nr < 2 || c.nz < 2 || c.nr > (1 << 20) || c.nz > (1 << 20) || c.n_xs < 2 || c.n_xs > (1 << 24))
    return PIC_EIO;
  const size_t nn = (size_t)(c.nr + 1) * (c.nz + 1), nc = (size_t)c.nr * c.nz;
  std::vector<int8_t> node(nn), cell(nc);
  std::vector<double> eps(nc), xe(c.n_xs), xsg(5 * (size_t)c.n_xs);
  F.get(node.data(), nn);
  F.get(cell.data(), nc);
  F.get(eps.data(), sizeof(double) * nc);
  F.get(xe.data(), sizeof(double) * xe.size());
  F.get(xsg.data(), sizeof(double) * xsg.size());
  int32_t host[2];
  F.get(host, sizeof(host));
  if (!F.ok) return PIC_EIO;
  c.node_kind = node.data();
  c.cell_kind = cell.data();
  c.cell_eps = eps.data();
  c.xs_energy = xe.data();
  c.xs_sigma = xsg.data();
  pic_handle *h = nullptr;
  int st = pic_init(&c, cuda_stream, &h);
  if (st) return st;
  st = [&]() -> int {
    int r;
    for (const Blob &b : state_blobs(h))
      if ((r = get_dev(F, b.p, b.n))) return r;
    h->cur = 0;
    for (int s = 0; s < 2; ++s) {
      const Store &S = h->st[0][s];
      BinMeta m;
      F.get(&m, sizeof(m));
      if (!F.ok) return PIC_EIO;
      const size_t nb = sizeof(int) * h->nbins;
      if ((r = get_dev(F, S.start, nb)) || (r = get_dev(F, S.cap, nb)) || (r = get_dev(F, S.fill, nb))) return r;
      uint64_t used = 0;
      F.get(&used, sizeof(used));
      if (!F.ok || used != used_slots(h, s, m) || used > (uint64_t)h->capacity[s]) return PIC_EIO;
      for (const Blob &b : store_columns(h, S, used))
        if ((r = get_dev(F, b.p, b.n))) return r;
      if (cudaMemcpy(S.meta, &m, sizeof(m), cudaMemcpyHostToDevice) != cudaSuccess) return PIC_ECUDA;
    }
    char extra;
    if (fread(&extra, 1, 1, F.f) != 0) return PIC_EIO;  // trailing bytes: not this format
    h->step = (uint32_t)host[0];
    h->started = host[1] != 0;
    return PIC_OK;
  }();
  if (st) {
    pic_destroy(h);
    return st;
  }
  *out = h;
  return PIC_OK;
}

}  // extern "C"
