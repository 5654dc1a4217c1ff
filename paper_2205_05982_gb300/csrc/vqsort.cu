// Host driver of libvqsort.so: argument checks, workspace layout, the fixed
// launch sequence of one sort, options, statistics and per-kernel timing.
// Everything data-dependent runs on the device; the host never waits inside
// a sort call.
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "launch.h"
#include "networks.h"
#include "../../include/vqsort.h"

using namespace vq;

namespace {

// ---------------------------------------------------------------------------
// Key types.
// ---------------------------------------------------------------------------
int key_bytes(vq_dtype dt) {
  switch (dt) {
    case VQ_I16: case VQ_U16: return 2;
    case VQ_I32: case VQ_U32: case VQ_F32: return 4;
    case VQ_I64: case VQ_U64: case VQ_F64: return 8;
    case VQ_U128: case VQ_KV64: return 16;
  }
  return 0;
}

Codec codec_of(vq_dtype dt, int ascending) {
  Codec c;
  c.desc = ascending ? 0 : 1;
  switch (dt) {
    case VQ_I16: case VQ_I32: case VQ_I64: c.kind = 1; break;
    case VQ_F32: case VQ_F64: c.kind = 2; break;
    case VQ_KV64: c.kind = 3; break;
    default: c.kind = 0; break;
  }
  return c;
}

// ---------------------------------------------------------------------------
// Options.
// ---------------------------------------------------------------------------
std::mutex g_mu;
int64_t g_depth_limit = -1;
int64_t g_leaf_cutoff = 0;
int64_t g_seed = 0x22050598;
int64_t g_spin_limit = 1 << 22;
int64_t g_test_stall = 0;
int64_t g_tile_bytes = 0;     // 0: by key size (tile_cpt)
int64_t g_leaf_threads = 0;   // 0: 16 keys per thread at the cutoff
int64_t g_kway = 1;           // K-way levels for ranges of >= 4 x the leaf cutoff
int64_t g_host_direct = 0;    // host sorts: 1 = leaves store into pinned host arrays

// 16-byte chunks per thread of a partition tile window. Default: 64 KiB
// windows (3 blocks per SM) for 8- and 16-byte keys, 32 KiB (5 per SM) for
// narrower keys, whose K-way tiles are capped at 16 keys per thread and so
// gain nothing from the larger window.
int tile_cpt(int kb) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_tile_bytes == 0) return kb >= 8 ? 16 : 8;
  return g_tile_bytes == 16384 ? 4 : g_tile_bytes == 65536 ? 16 : 8;
}

// Tile windows of a sort of n keys in `segments` arrays: the option if set;
// else 16 KiB windows for one array of 4- or 8-byte keys short enough for
// the 16384-key leaf cutoff: its one K-way level has few tiles, and more,
// smaller tiles keep more of the grid busy (L2 flushed: 1e6 u64 keys
// 151 -> 131 us, 2.5e5 127 -> 106 us, 1e6 u32 118 -> 102 us). 2-byte keys'
// K-way tiles are the same size in 16 and 32 KiB windows, so they keep the
// per-key-size default, as do 16-byte keys.
int sort_tile_cpt(int kb, uint64_t n, uint64_t segments) {
  bool opt;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    opt = g_tile_bytes != 0;
  }
  if (!opt && (kmem(kb) == 4 || kmem(kb) == 8) && size_leaf_cutoff(kb, n, segments) == 16384u) return 4;
  return tile_cpt(kb);
}

// Library-owned workspaces are sized for the smallest tile window (the
// largest work queue), like vqsort_workspace_bytes, so they cover whichever
// window a sort takes.
constexpr int OWNED_WS_CPT = 4;

// The leaf cutoff of a sort of n keys in `segments` arrays: the option if
// set, else the size rule.
unsigned leaf_cutoff_for(int kb, uint64_t n, uint64_t segments) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_leaf_cutoff > 0) return (unsigned)g_leaf_cutoff < max_leaf_cutoff(kb) ? (unsigned)g_leaf_cutoff
                                                                             : max_leaf_cutoff(kb);
  const unsigned c = size_leaf_cutoff(kb, n, segments);
  return c < max_leaf_cutoff(kb) ? c : max_leaf_cutoff(kb);
}

// ---------------------------------------------------------------------------
// Workspace layout.
// ---------------------------------------------------------------------------
struct Layout {
  size_t hdr, segs, items, lw, lm, lb, fb, kw, ids, alt, total;
  unsigned cap_q, cap_segs, cap_lw, cap_lm, cap_lb, cap_fb, cap_kw;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout make_layout(int kb, uint64_t n, uint64_t S, unsigned C, int64_t depth_limit, bool with_alt,
                   int cpt) {
  const uint64_t lg = floor_log2_u64(n < 2 ? 2 : n);
  uint64_t levels = 2 * lg + 4;
  if (depth_limit >= 0 && (uint64_t)depth_limit > levels) levels = (uint64_t)depth_limit;
  levels += 2;
  const uint64_t per_level = n / (C + 1ull) + 1;
  Layout L{};
  const uint64_t cap_segs = (levels + 1) * per_level + 16;
  // Per level: a K-way range runs its scatter tiles (T_K keys, half a
  // window) and half as many counting tiles, bounded here by two passes of
  // scatter tiles; every range may add a partial tile per pass and one setup
  // item.
  const uint64_t TK = kw_tile_keys(kb, cpt);
  const uint64_t cap_q = (levels + 1) * (2 * (n / TK + 1) + 3 * per_level) + 2 * S + 16;
  // K-way records: ranges of >= 4C keys; when they run out, ranges are split
  // in two instead
  const uint64_t cap_kw = 2 * (n / (4ull * C) + 1) + 64;
  const uint64_t cap_lw = 2 * cap_segs + S + 16;
  const uint64_t cap_lm = n / (WARP_LEAF_MAX + 1) + S + 16;   // mid leaves hold > 512 keys each
  const uint64_t cap_lb = n / 512 + n / C + 2 * cap_segs + S + 16;
  const uint64_t cap_fb = n / (C + 1ull) + S + 16;
  L.cap_segs = (unsigned)cap_segs;
  L.cap_q = (unsigned)cap_q;
  L.cap_lw = (unsigned)cap_lw;
  L.cap_lm = (unsigned)cap_lm;
  L.cap_lb = (unsigned)cap_lb;
  L.cap_fb = (unsigned)cap_fb;
  L.cap_kw = (unsigned)cap_kw;
  size_t off = 0;
  L.hdr = off; off = align256(off + sizeof(Header));
  L.segs = off; off = align256(off + cap_segs * sizeof(SegDesc));
  L.items = off; off = align256(off + cap_q * 8);
  L.lw = off; off = align256(off + cap_lw * sizeof(LeafEntry));
  L.lm = off; off = align256(off + cap_lm * sizeof(LeafEntry));
  L.lb = off; off = align256(off + cap_lb * sizeof(LeafEntry));
  L.fb = off; off = align256(off + cap_fb * sizeof(LeafEntry));
  L.kw = off; off = align256(off + cap_kw * sizeof(KwayDesc));
  L.ids = off; off = align256(off + n + 16);
  L.alt = off;
  if (with_alt) off = align256(off + n * (uint64_t)kb);
  L.total = off;
  return L;
}

// ---------------------------------------------------------------------------
// Library-owned workspaces, one per (device, stream).
// ---------------------------------------------------------------------------
struct OwnedWs {
  void *ptr = nullptr;
  size_t bytes = 0;
};
std::map<std::pair<int, cudaStream_t>, OwnedWs> g_ws;

vq_status owned_ws(cudaStream_t s, size_t need, void **ptr, size_t *bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VQ_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  OwnedWs &w = g_ws[{dev, s}];
  if (w.bytes < need) {
    if (w.ptr) {
      if (cudaStreamSynchronize(s) != cudaSuccess) return VQ_ERR_CUDA;
      cudaFree(w.ptr);
      w.ptr = nullptr;
      w.bytes = 0;
    }
    const size_t grow = need + need / 8;
    if (cudaMalloc(&w.ptr, grow) != cudaSuccess) {
      cudaGetLastError();
      return VQ_ERR_NOMEM;
    }
    w.bytes = grow;
  }
  *ptr = w.ptr;
  *bytes = w.bytes;
  return VQ_OK;
}

const void *lookup_ws(cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_ws.find({dev, s});
  return it == g_ws.end() ? nullptr : it->second.ptr;
}

// ---------------------------------------------------------------------------
// Side streams of the leaf kernels, one pair per (device, stream). After the
// partition the leaf kernels write disjoint ranges and never wait on one
// another, so two of them run on side streams that fork from the caller's
// stream and join it again through events (a CUDA-graph capture of the
// caller's stream takes the fork and the join in as well). Created on the
// first sort on a stream that is not being captured; until then, and if
// creation fails, the leaf kernels run one after another on the caller's
// stream.
// ---------------------------------------------------------------------------
struct Fork {
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
  std::mutex mu;   // one fork/join sequence at a time per caller stream
};
std::map<std::pair<int, cudaStream_t>, std::unique_ptr<Fork>> g_fork;

Fork *fork_for(cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  std::unique_ptr<Fork> &f = g_fork[{dev, s}];
  if (f) return f.get();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return nullptr;
  }
  // the side streams take the caller's stream priority, so that a
  // high-priority sort stays high-priority through its leaf phase
  int prio = 0;
  if (cudaStreamGetPriority(s, &prio) != cudaSuccess) {
    cudaGetLastError();
    prio = 0;
  }
  auto nf = std::make_unique<Fork>();
  bool ok = cudaEventCreateWithFlags(&nf->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < 2 && ok; ++i) {
    ok = cudaStreamCreateWithPriority(&nf->side[i], cudaStreamNonBlocking, prio) == cudaSuccess &&
         cudaEventCreateWithFlags(&nf->join[i], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    for (int i = 0; i < 2; ++i) {
      if (nf->side[i]) cudaStreamDestroy(nf->side[i]);
      if (nf->join[i]) cudaEventDestroy(nf->join[i]);
    }
    if (nf->fork) cudaEventDestroy(nf->fork);
    return nullptr;
  }
  f = std::move(nf);
  return f.get();
}

// ---------------------------------------------------------------------------
// Per-kernel timing.
// ---------------------------------------------------------------------------
struct ProfEntry {
  double ms = 0;
  uint64_t launches = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
bool g_prof = false;
std::map<std::string, ProfEntry> g_prof_tab;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

template <class F> cudaError_t timed(const char *name, cudaStream_t s, F &&f) {
  bool prof;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    prof = g_prof;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (prof) cudaStreamIsCapturing(s, &cs);
  if (!prof || cs != cudaStreamCaptureStatusNone) return f();
  cudaEvent_t e0, e1;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    e0 = take_event();
    e1 = take_event();
  }
  cudaEventRecord(e0, s);
  const cudaError_t err = f();
  cudaEventRecord(e1, s);
  std::lock_guard<std::mutex> lk(g_mu);
  ProfEntry &p = g_prof_tab[name];
  p.pending.push_back({e0, e1});
  p.launches++;
  return err;
}

// ---------------------------------------------------------------------------
// Device check (compute capability 10.3).
// ---------------------------------------------------------------------------
vq_status check_device() {
  static int ok_dev = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VQ_ERR_CUDA;
  if (ok_dev == dev) return VQ_OK;
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
    return VQ_ERR_CUDA;
  if (major != 10 || minor != 3) return VQ_ERR_UNSUPPORTED;
  ok_dev = dev;
  return VQ_OK;
}

vq_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VQ_OK : VQ_ERR_CUDA; }

// ---------------------------------------------------------------------------
// One sort (or one standalone partition) on a workspace.
// ---------------------------------------------------------------------------
struct Job {
  vq_dtype dt;
  void *keys;
  void *alt_given;                 // MODE_PARTITION: the output buffer
  uint64_t n;
  const uint64_t *offsets;
  uint64_t num_segments;
  int ascending;
  unsigned mode;
  const void *pivot_host;
  uint64_t *out_left;
  void *out = nullptr;             // sorted keys go here (default: keys)
  int kclass = 0;                  // kernel key class (0: the key bytes; KV_KEYONLY: pairs by key)
};

vq_status run(const Job &j, void *ws, size_t ws_bytes, cudaStream_t s) {
  const int kb = key_bytes(j.dt);
  const unsigned C = leaf_cutoff_for(kb, j.n, j.num_segments);
  int64_t depth_limit, seed, spin, stall, leaf_threads, kway;
  const int cpt = j.mode == MODE_SORT ? sort_tile_cpt(kb, j.n, j.num_segments) : tile_cpt(kb);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    depth_limit = g_depth_limit;
    seed = g_seed;
    spin = g_spin_limit;
    stall = g_test_stall;
    leaf_threads = g_leaf_threads;
    kway = g_kway;
  }
  const bool with_alt = j.mode == MODE_SORT;
  const Layout L = make_layout(kb, j.n, j.num_segments, C, depth_limit, with_alt, cpt);
  if (!ws || ws_bytes < L.total) return VQ_ERR_NOMEM;
  if ((uintptr_t)ws & 255) return VQ_ERR_INVALID;
  unsigned char *w = (unsigned char *)ws;
  SortArgs a{};
  a.keys = j.keys;
  a.out = j.out ? j.out : j.keys;
  a.alt = with_alt ? (void *)(w + L.alt) : j.alt_given;
  a.hdr = (Header *)(w + L.hdr);
  a.segs = (SegDesc *)(w + L.segs);
  a.items = (unsigned long long *)(w + L.items);
  a.leaf_warp = (LeafEntry *)(w + L.lw);
  a.leaf_mid = (LeafEntry *)(w + L.lm);
  a.leaf_block = (LeafEntry *)(w + L.lb);
  a.fb = (LeafEntry *)(w + L.fb);
  a.kw = (kway && j.mode == MODE_SORT) ? (KwayDesc *)(w + L.kw) : nullptr;
  a.kw_ids = w + L.ids;
  a.cap_kw = L.cap_kw;
  a.offsets = (const unsigned long long *)j.offsets;
  a.n_total = j.n;
  a.num_segments = j.num_segments;
  a.out_left = (unsigned long long *)j.out_left;
  a.seed = (unsigned long long)seed;
  a.cap_q = L.cap_q;
  a.cap_segs = L.cap_segs;
  a.cap_leaf_warp = L.cap_lw;
  a.cap_leaf_mid = L.cap_lm;
  a.mid_max = mid_leaf_limit(kb);
  a.cap_leaf_block = L.cap_lb;
  a.cap_fb = L.cap_fb;
  a.tile_keys = part_tile_keys(kb, cpt);
  a.kw_tile_keys = kw_tile_keys(kb, cpt);
  a.kw_min_keys = 4 * C;
  a.kw_target = C / 4;
  a.tile_cpt = (unsigned)cpt;
  a.leaf_threads = (unsigned)leaf_threads;   // 16-byte keys: 256 or (default) 512
  a.leaf_cutoff = C;
  a.depth_override = (int)depth_limit;
  a.spin_limit = (unsigned)spin;
  a.mode = j.mode;
  a.test_stall = (unsigned)stall;
  a.codec = codec_of(j.dt, j.ascending);
  a.pivot = U128{0, 0};
  if (j.mode == MODE_PARTITION) {
    // the pivot's code, by the same codec the kernels use
    switch (kb) {
      case 2: { uint16_t v; memcpy(&v, j.pivot_host, 2); a.pivot.lo = encode<2>(v, a.codec); break; }
      case 4: { uint32_t v; memcpy(&v, j.pivot_host, 4); a.pivot.lo = encode<4>(v, a.codec); break; }
      case 8: { uint64_t v; memcpy(&v, j.pivot_host, 8); a.pivot.lo = encode<8>(v, a.codec); break; }
      case 16: { U128 v; memcpy(&v, j.pivot_host, 16); a.pivot = encode<16>(v, a.codec); break; }
    }
  }
  cudaError_t e;
  const int kc = j.kclass ? j.kclass : kb;
  if ((e = timed("prep", s, [&] { return launch_prep(a, s); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed("seed", s, [&] { return launch_seed(kc, a, s); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed("partition", s, [&] { return launch_partition(kc, a, s); })) != cudaSuccess) return cuda_status(e);
  if (j.mode == MODE_SORT) {
    // the leaf phase, timed as a whole ("leaves") as well as per kernel:
    // with the fork its kernels overlap
    Fork *fk = fork_for(s);
    e = timed("leaves", s, [&]() -> cudaError_t {
      cudaError_t x;
      if (!fk) {
        if ((x = timed("leaf_warp", s, [&] { return launch_leaf_warp(kc, a, s); })) != cudaSuccess) return x;
        if ((x = timed("leaf_mid", s, [&] { return launch_leaf_mid(kc, a, s); })) != cudaSuccess) return x;
        return timed("leaf_block", s, [&] { return launch_leaf_block(kc, a, s); });
      }
      // block leaves and warp leaves on the side streams, mid leaves here;
      // the join is enqueued even when a launch failed
      std::lock_guard<std::mutex> flk(fk->mu);
      cudaStream_t b = fk->side[0], w = fk->side[1];
      x = cudaEventRecord(fk->fork, s);
      if (x == cudaSuccess) x = cudaStreamWaitEvent(b, fk->fork, 0);
      if (x == cudaSuccess) x = cudaStreamWaitEvent(w, fk->fork, 0);
      if (x != cudaSuccess) return x;
      const cudaError_t eb = timed("leaf_block", b, [&] { return launch_leaf_block(kc, a, b); });
      const cudaError_t ew = timed("leaf_warp", w, [&] { return launch_leaf_warp(kc, a, w); });
      const cudaError_t em = timed("leaf_mid", s, [&] { return launch_leaf_mid(kc, a, s); });
      x = cudaEventRecord(fk->join[0], b);
      if (x == cudaSuccess) x = cudaEventRecord(fk->join[1], w);
      if (x == cudaSuccess) x = cudaStreamWaitEvent(s, fk->join[0], 0);
      if (x == cudaSuccess) x = cudaStreamWaitEvent(s, fk->join[1], 0);
      for (cudaError_t y : {eb, ew, em})
        if (y != cudaSuccess) return y;
      return x;
    });
    if (e != cudaSuccess) return cuda_status(e);
    // cooperative (its blocks must be resident together): after the join
    if ((e = timed("fallback", s, [&] { return launch_fallback(kc, a, s); })) != cudaSuccess) return cuda_status(e);
  }
  return VQ_OK;
}

vq_status check_keys(vq_dtype dt, const void *p, uint64_t n) {
  const int kb = key_bytes(dt);
  if (!kb) return VQ_ERR_INVALID;
  if (n > 0 && !p) return VQ_ERR_INVALID;
  if ((uintptr_t)p % kb) return VQ_ERR_INVALID;
  if (n >= (1ull << 32) - 1) return VQ_ERR_INVALID;   // per-range lengths are 32-bit in leaf lists
  return VQ_OK;
}

vq_status sort_common(vq_dtype dt, void *keys, uint64_t n, const uint64_t *offsets, uint64_t S, int asc,
                      void *ws, size_t ws_bytes, void *stream, int kclass = 0) {
  vq_status st = check_keys(dt, keys, n);
  if (st != VQ_OK) return st;
  if (offsets == nullptr && n <= 1) return VQ_OK;
  if (offsets != nullptr && S == 0) return VQ_OK;
  if ((st = check_device()) != VQ_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (!ws) {
    const int kb = key_bytes(dt);
    int64_t dl;
    {
      std::lock_guard<std::mutex> lk(g_mu);
      dl = g_depth_limit;
    }
    const uint64_t nseg = offsets ? S : 1;
    const Layout L = make_layout(kb, n, nseg, leaf_cutoff_for(kb, n, nseg), dl, true, OWNED_WS_CPT);
    if ((st = owned_ws(s, L.total, &ws, &ws_bytes)) != VQ_OK) return st;
  }
  Job j{dt, keys, nullptr, n, offsets, offsets ? S : 1, asc, MODE_SORT, nullptr, nullptr};
  j.kclass = kclass;
  return run(j, ws, ws_bytes, s);
}

// Library-owned resources of the host entry point.
struct HostCtx {
  cudaStream_t stream = nullptr;
};
std::map<int, HostCtx> g_host;
// Device copies of host arrays, one per (device, stream).
struct DevBuf {
  void *ptr = nullptr;
  size_t bytes = 0;
};
std::map<std::pair<int, cudaStream_t>, DevBuf> g_hostbuf;

vq_status read_header(const void *ws, void *stream, Header *h) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!ws) {
    ws = lookup_ws(s);
    if (!ws) {   // no sort has used the library's workspace on this stream yet
      memset(h, 0, sizeof(Header));
      return VQ_OK;
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return VQ_ERR_CUDA;
  if (cudaMemcpy(h, ws, sizeof(Header), cudaMemcpyDeviceToHost) != cudaSuccess) return VQ_ERR_CUDA;
  return VQ_OK;
}

// Uploads a host array to a device buffer owned for (device, stream), sorts
// it and brings the keys back, all enqueued on `s`; nothing waits. A pinned
// (page-locked, mapped) host array is written by the leaf kernels
// themselves, so the download runs during the leaves' network work instead
// of after it; other host memory is copied back after the sort.
vq_status host_enqueue(vq_dtype dt, void *h_keys, size_t n, int ascending, cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VQ_ERR_CUDA;
  const int kb = key_bytes(dt);
  const size_t bytes = n * (size_t)kb;
  void *dbuf = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    DevBuf &b = g_hostbuf[{dev, s}];
    if (b.bytes < bytes) {
      if (b.ptr) cudaFree(b.ptr);
      b.ptr = nullptr;
      b.bytes = 0;
      if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        return VQ_ERR_NOMEM;
      }
      b.bytes = bytes;
    }
    dbuf = b.ptr;
  }
  int64_t dl, direct;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    dl = g_depth_limit;
    direct = g_host_direct;
  }
  // a pinned array is written by the leaves themselves (unless the option
  // asks for a copy back), so its download overlaps their work
  void *h_dev = nullptr;
  cudaPointerAttributes attr{};
  if (direct && cudaPointerGetAttributes(&attr, h_keys) == cudaSuccess &&
      attr.type == cudaMemoryTypeHost && attr.devicePointer)
    h_dev = attr.devicePointer;
  cudaGetLastError();
  if (cudaMemcpyAsync(dbuf, h_keys, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return VQ_ERR_CUDA;
  const Layout L = make_layout(kb, n, 1, leaf_cutoff_for(kb, n, 1), dl, true, OWNED_WS_CPT);
  void *ws;
  size_t wsb;
  vq_status st;
  if ((st = owned_ws(s, L.total, &ws, &wsb)) != VQ_OK) return st;
  Job j{dt, dbuf, nullptr, n, nullptr, 1, ascending, MODE_SORT, nullptr, nullptr};
  j.out = h_dev;
  if ((st = run(j, ws, wsb, s)) != VQ_OK) return st;
  if (!h_dev && cudaMemcpyAsync(h_keys, dbuf, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return VQ_ERR_CUDA;
  return VQ_OK;
}

}  // namespace

extern "C" {

vq_status vqsort_sort(vq_dtype dt, void *d_keys, size_t n, int ascending, void *stream) {
  return sort_common(dt, d_keys, n, nullptr, 1, ascending, nullptr, 0, stream);
}

vq_status vqsort_sort_kv(void *d_pairs, size_t n, int ascending, void *stream) {
  return sort_common(VQ_KV64, d_pairs, n, nullptr, 1, ascending, nullptr, 0, stream);
}

vq_status vqsort_sort_kv_by_key(void *d_pairs, size_t n, int ascending, void *stream) {
  return sort_common(VQ_KV64, d_pairs, n, nullptr, 1, ascending, nullptr, 0, stream, KV_KEYONLY);
}

vq_status vqsort_sort_kv_by_key_ws(void *d_pairs, size_t n, int ascending, void *d_ws, size_t ws_bytes,
                                   void *stream) {
  if (!d_ws) return VQ_ERR_INVALID;
  return sort_common(VQ_KV64, d_pairs, n, nullptr, 1, ascending, d_ws, ws_bytes, stream, KV_KEYONLY);
}

vq_status vqsort_sort_segmented(vq_dtype dt, void *d_keys, size_t n_total, const uint64_t *d_offsets,
                                size_t num_segments, int ascending, void *stream) {
  if (!d_offsets && num_segments) return VQ_ERR_INVALID;
  return sort_common(dt, d_keys, n_total, d_offsets, num_segments, ascending, nullptr, 0, stream);
}

size_t vqsort_workspace_bytes(vq_dtype dt, size_t n_total, size_t num_segments) {
  const int kb = key_bytes(dt);
  if (!kb) return 0;
  int64_t dl;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    dl = g_depth_limit;
  }
  const uint64_t S = num_segments ? num_segments : 1;
  return make_layout(kb, n_total, S, leaf_cutoff_for(kb, n_total, S), dl, true, OWNED_WS_CPT).total;
}

vq_status vqsort_sort_ws(vq_dtype dt, void *d_keys, size_t n, int ascending, void *d_ws, size_t ws_bytes,
                         void *stream) {
  if (!d_ws) return VQ_ERR_INVALID;
  return sort_common(dt, d_keys, n, nullptr, 1, ascending, d_ws, ws_bytes, stream);
}

vq_status vqsort_sort_segmented_ws(vq_dtype dt, void *d_keys, size_t n_total, const uint64_t *d_offsets,
                                   size_t num_segments, int ascending, void *d_ws, size_t ws_bytes,
                                   void *stream) {
  if (!d_ws || (!d_offsets && num_segments)) return VQ_ERR_INVALID;
  return sort_common(dt, d_keys, n_total, d_offsets, num_segments, ascending, d_ws, ws_bytes, stream);
}

vq_status vqsort_sort_host(vq_dtype dt, void *h_keys, size_t n, int ascending) {
  vq_status st = check_keys(dt, h_keys, n);
  if (st != VQ_OK) return st;
  if (n <= 1) return VQ_OK;
  if ((st = check_device()) != VQ_OK) return st;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaStream_t s;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    HostCtx &hc = g_host[dev];
    if (!hc.stream && cudaStreamCreateWithFlags(&hc.stream, cudaStreamNonBlocking) != cudaSuccess)
      return VQ_ERR_CUDA;
    s = hc.stream;
  }
  if ((st = host_enqueue(dt, h_keys, n, ascending, s)) != VQ_OK) return st;
  return vqsort_last_device_status(nullptr, s);
}

vq_status vqsort_sort_host_async(vq_dtype dt, void *h_keys, size_t n, int ascending, void *stream) {
  vq_status st = check_keys(dt, h_keys, n);
  if (st != VQ_OK) return st;
  if (n <= 1) return VQ_OK;
  if ((st = check_device()) != VQ_OK) return st;
  return host_enqueue(dt, h_keys, n, ascending, (cudaStream_t)stream);
}

vq_status vqsort_partition(vq_dtype dt, const void *d_in, void *d_out, size_t n, const void *h_pivot,
                           int ascending, uint64_t *d_left_count, void *stream) {
  vq_status st = check_keys(dt, d_in, n);
  if (st != VQ_OK) return st;
  if ((st = check_keys(dt, d_out, n)) != VQ_OK) return st;
  if (!h_pivot || !d_left_count || (n > 0 && d_in == d_out)) return VQ_ERR_INVALID;
  if ((st = check_device()) != VQ_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int kb = key_bytes(dt);
  const Layout L = make_layout(kb, n, 1, leaf_cutoff_for(kb, n, 1), -1, false, tile_cpt(kb));
  void *ws;
  size_t wsb;
  if ((st = owned_ws(s, L.total, &ws, &wsb)) != VQ_OK) return st;
  Job j{dt, const_cast<void *>(d_in), d_out, n, nullptr, 1, ascending, MODE_PARTITION, h_pivot, d_left_count};
  return run(j, ws, wsb, s);
}

vq_status vqsort_sort_stable(vq_dtype dt, void *d_keys, size_t n, int ascending, uint64_t *d_rows,
                             void *stream) {
  vq_status st = check_keys(dt, d_keys, n);
  if (st != VQ_OK) return st;
  const int kb = key_bytes(dt);
  if (kb == 16) return VQ_ERR_UNSUPPORTED;
  if (n > 0 && (!d_rows || ((uintptr_t)d_rows & 7))) return VQ_ERR_INVALID;
  if (n == 0) return VQ_OK;
  if ((st = check_device()) != VQ_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // packed codes: 8 bytes for keys of up to 4 bytes, 16 for 8-byte keys
  const vq_dtype pdt = kb == 8 ? VQ_U128 : VQ_U64;
  const int pkb = key_bytes(pdt);
  int64_t dl;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    dl = g_depth_limit;
  }
  const Layout L = make_layout(pkb, n, 1, leaf_cutoff_for(pkb, n, 1), dl, true, OWNED_WS_CPT);
  const size_t packed_off = align256(L.total);
  void *ws;
  size_t wsb;
  if ((st = owned_ws(s, packed_off + (size_t)n * pkb, &ws, &wsb)) != VQ_OK) return st;
  void *packed = (unsigned char *)ws + packed_off;
  const Codec cd = codec_of(dt, ascending);
  cudaError_t e;
  if ((e = timed("stable_pack", s, [&] { return launch_stable_pack(kb, d_keys, packed, n, cd, s); })) !=
      cudaSuccess)
    return cuda_status(e);
  if (n > 1) {
    Job j{pdt, packed, nullptr, n, nullptr, 1, 1, MODE_SORT, nullptr, nullptr};
    if ((st = run(j, ws, packed_off, s)) != VQ_OK) return st;
  }
  if ((e = timed("stable_unpack", s, [&] { return launch_stable_unpack(kb, packed, d_keys, d_rows, n, cd, s); })) !=
      cudaSuccess)
    return cuda_status(e);
  return VQ_OK;
}

vq_status vqsort_choose_pivot(vq_dtype dt, const void *d_keys, size_t n, uint64_t seed, int ascending,
                              void *d_pivot_out, void *stream) {
  vq_status st = check_keys(dt, d_keys, n);
  if (st != VQ_OK) return st;
  if (n < 1024 || !d_pivot_out) return VQ_ERR_INVALID;
  if ((st = check_device()) != VQ_OK) return st;
  SortArgs a{};
  a.codec = codec_of(dt, ascending);
  cudaStream_t s = (cudaStream_t)stream;
  return cuda_status(timed("choose_pivot", s, [&] {
    return launch_choose_pivot(key_bytes(dt), a, d_keys, n, seed, d_pivot_out, s);
  }));
}

vq_status vqsort_last_device_status(const void *d_ws, void *stream) {
  Header h;
  const vq_status st = read_header(d_ws, stream, &h);
  if (st != VQ_OK) return st;
  return (vq_status)h.error;
}

vq_status vqsort_device_status_async(const void *d_ws, uint64_t *h_status, void *stream) {
  if (!d_ws || !h_status) return VQ_ERR_INVALID;
  const Header *h = (const Header *)d_ws;
  return cuda_status(cudaMemcpyAsync(h_status, &h->error, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                     (cudaStream_t)stream));
}

vq_status vqsort_release_stream(void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VQ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return VQ_ERR_CUDA;
  std::unique_ptr<Fork> f;
  OwnedWs w;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_fork.find({dev, s});
    if (it != g_fork.end()) {
      f = std::move(it->second);
      g_fork.erase(it);
    }
    auto jt = g_ws.find({dev, s});
    if (jt != g_ws.end()) {
      w = jt->second;
      g_ws.erase(jt);
    }
  }
  bool ok = true;
  if (f) {
    // the joins the stream waited for mean the side streams are idle too
    for (int i = 0; i < 2; ++i) {
      ok = cudaStreamDestroy(f->side[i]) == cudaSuccess && ok;
      ok = cudaEventDestroy(f->join[i]) == cudaSuccess && ok;
    }
    ok = cudaEventDestroy(f->fork) == cudaSuccess && ok;
  }
  if (w.ptr) ok = cudaFree(w.ptr) == cudaSuccess && ok;
  return ok ? VQ_OK : VQ_ERR_CUDA;
}

vq_status vqsort_get_stats(const void *d_ws, void *stream, vq_stats *out) {
  if (!out) return VQ_ERR_INVALID;
  Header h;
  const vq_status st = read_header(d_ws, stream, &h);
  if (st != VQ_OK) return st;
  out->keys_partitioned = h.keys_partitioned;
  out->tiles = h.tiles;
  out->segments = h.segments;
  out->leaves_warp = h.leaves_warp;
  out->leaves_block = h.leaves_block;
  out->leaf_keys = h.leaf_keys;
  out->equal_ranges = h.equal_ranges;
  out->equal_keys = h.equal_keys;
  out->degenerate = h.degenerate;
  out->fallback_ranges = h.fallback_ranges;
  out->fallback_keys = h.fallback_keys;
  out->max_depth = h.max_depth;
  out->keys_counted = h.keys_counted;
  out->kway_ranges = h.kway_ranges;
  out->guard = h.guard;
  out->partition_blocks = h.part_grid;
  out->leaves_mid = h.leaves_mid;
  out->leaf_ce = h.leaf_ce;
  out->leaf_keys_warp = h.leaf_keys_warp;
  out->leaf_keys_mid = h.leaf_keys_mid;
  out->leaf_keys_block = h.leaf_keys_block;
  out->device_status = h.error;
  return VQ_OK;
}

const char *vqsort_status_string(vq_status s) {
  switch (s) {
    case VQ_OK: return "ok";
    case VQ_ERR_INVALID: return "invalid argument";
    case VQ_ERR_UNSUPPORTED: return "unsupported device (needs compute capability 10.3)";
    case VQ_ERR_NOMEM: return "workspace too small or allocation failed";
    case VQ_ERR_CUDA: return "CUDA runtime error";
    case VQ_ERR_TIMEOUT: return "a bounded device-side wait ran out";
    case VQ_ERR_INTERNAL: return "device-side capacity overflow";
  }
  return "unknown status";
}

vq_status vqsort_set_option(vq_option opt, int64_t value) {
  std::lock_guard<std::mutex> lk(g_mu);
  switch (opt) {
    case VQ_OPT_DEPTH_LIMIT:
      if (value < -1 || value > 1000) return VQ_ERR_INVALID;
      g_depth_limit = value;
      return VQ_OK;
    case VQ_OPT_LEAF_CUTOFF:
      // applies to every key size; 16-byte keys clamp it to 4096
      if (value != 0 && (value < 1024 || value > 16384 || (value & (value - 1)))) return VQ_ERR_INVALID;
      g_leaf_cutoff = value;
      return VQ_OK;
    case VQ_OPT_SEED: g_seed = value; return VQ_OK;
    case VQ_OPT_SPIN_LIMIT:
      if (value < 1 || value > (1ll << 30)) return VQ_ERR_INVALID;
      g_spin_limit = value;
      return VQ_OK;
    case VQ_OPT_TEST_STALL: g_test_stall = value ? 1 : 0; return VQ_OK;
    case VQ_OPT_TILE_BYTES:
      if (value != 0 && value != 16384 && value != 32768 && value != 65536) return VQ_ERR_INVALID;
      g_tile_bytes = value;
      return VQ_OK;
    case VQ_OPT_LEAF_THREADS:
      if (value != 0 && value != 256 && value != 512 && value != 1024) return VQ_ERR_INVALID;
      g_leaf_threads = value;
      return VQ_OK;
    case VQ_OPT_KWAY: g_kway = value ? 1 : 0; return VQ_OK;
    case VQ_OPT_HOST_DIRECT: g_host_direct = value ? 1 : 0; return VQ_OK;
  }
  return VQ_ERR_INVALID;
}

int64_t vqsort_get_option(vq_option opt) {
  std::lock_guard<std::mutex> lk(g_mu);
  switch (opt) {
    case VQ_OPT_DEPTH_LIMIT: return g_depth_limit;
    case VQ_OPT_LEAF_CUTOFF: return g_leaf_cutoff;
    case VQ_OPT_SEED: return g_seed;
    case VQ_OPT_SPIN_LIMIT: return g_spin_limit;
    case VQ_OPT_TEST_STALL: return g_test_stall;
    case VQ_OPT_TILE_BYTES: return g_tile_bytes;
    case VQ_OPT_LEAF_THREADS: return g_leaf_threads;
    case VQ_OPT_KWAY: return g_kway;
    case VQ_OPT_HOST_DIRECT: return g_host_direct;
  }
  return -1;
}

vq_status vqsort_merge_schedule(unsigned run_len, unsigned keys_per_thread, unsigned *pairs_out, size_t max_pairs,
                                size_t *n_pairs) {
  const unsigned L = run_len, R = keys_per_thread;
  if (!n_pairs || L == 0 || R == 0 || (L & (L - 1)) || (R & (R - 1)) || R > L) return VQ_ERR_INVALID;
  size_t k = 0;
  const unsigned steps = vq_merge_steps(L);
  for (unsigned s = 0; s < steps; ++s) {
    const VqMergeStep m = vq_merge_step(L, R, s);
    for (unsigned t = 0; t < 2 * L / R; ++t) {
      for (unsigned r = 0; r < R; ++r) {
        unsigned pt, pr;
        if (m.lane_xor) {
          pt = t ^ m.lane_xor;
          pr = m.reverse ? R - 1 - r : r;
        } else {
          pt = t;
          pr = r ^ m.reg_xor;
        }
        const unsigned i = t * R + r, j = pt * R + pr;
        if (i < j) {
          if (pairs_out && k < max_pairs) {
            pairs_out[2 * k] = i;
            pairs_out[2 * k + 1] = j;
          }
          ++k;
        }
      }
    }
  }
  *n_pairs = k;
  return VQ_OK;
}

vq_status vqsort_profile_enable(int enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_prof = enable != 0;
  return VQ_OK;
}

vq_status vqsort_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &kv : g_prof_tab)
    for (auto &pe : kv.second.pending) {
      cudaEventSynchronize(pe.second);
      g_event_pool.push_back(pe.first);
      g_event_pool.push_back(pe.second);
    }
  g_prof_tab.clear();
  return VQ_OK;
}

vq_status vqsort_profile_read(const char **names, double *ms, uint64_t *launches, size_t max, size_t *count) {
  std::lock_guard<std::mutex> lk(g_mu);
  size_t k = 0;
  for (auto &kv : g_prof_tab) {
    ProfEntry &p = kv.second;
    for (auto &pe : p.pending) {
      if (cudaEventSynchronize(pe.second) != cudaSuccess) return VQ_ERR_CUDA;
      float t = 0;
      cudaEventElapsedTime(&t, pe.first, pe.second);
      p.ms += t;
      g_event_pool.push_back(pe.first);
      g_event_pool.push_back(pe.second);
    }
    p.pending.clear();
    if (k < max) {
      if (names) names[k] = kv.first.c_str();
      if (ms) ms[k] = p.ms;
      if (launches) launches[k] = p.launches;
    }
    ++k;
  }
  if (count) *count = k;
  return VQ_OK;
}

}  // extern "C"
