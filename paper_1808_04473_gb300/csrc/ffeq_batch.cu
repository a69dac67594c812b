// Uneven batches (include/ffeq_batch.h): host-side schedule and launches.
//
// Every (instance, subcarrier) becomes one unit of work with a BatchDesc.
// Units are grouped by users padded to 8/16/32 (the register shape of both
// kernels); a group whose shared-memory capacities would not fit together is
// split.  Per group:
//   * the contraction kernel runs persistently on min(units, #SMs) CTAs and
//     takes units from a device work queue; the group's descriptors are stored
//     in decreasing order of cost ((U + n_sym) * B complex to stage), so the
//     queue hands out the largest units first (longest-processing-time order);
//   * the solve/fusion kernel packs units into tiles of at most
//     threads / (UP * lanes per row) local systems (next fit over units sorted
//     by decreasing Ceff), one CTA per tile.
// The tables live in page-locked host memory and are copied into the front of
// the caller's workspace; the device checks every descriptor against the
// buffer extents before using it.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ffeq_batch.h"
#include "ffeq_internal.h"

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxGroups = 64;                // queue counters in the first 256 bytes
constexpr size_t kSolveSmemLimit = 227 * 1024;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

struct Group {
  int UP;
  int max_ceff;           // largest Ceff of a unit in the group
  bool bulk_ok;           // every unit: even B and 16-byte aligned row offsets
  int stage_elems, slot_elems, n_slots, max_stages;
  // tuning
  int stages, threads, lpr;
  // tables (indices into the batch-wide arrays)
  long long first, n_units;       // descriptors [first, first + n_units) in both orders
  long long tile_first, n_tiles;  // tiles of this group
};

}  // namespace

struct ffeq_batch {
  ffeq_batch_config cfg;
  int n_inst = 0;
  long long n_units = 0;
  std::vector<ffeq::BatchDesc> units;       // instance order
  std::vector<Group> groups;
  std::vector<long long> gram_order, solve_order;   // per group ranges, unit indices
  // page-locked table image: [counters][gram desc][solve desc][tiles][slot maps]
  unsigned char* host = nullptr;
  size_t off_gram = 0, off_solve = 0, off_tiles = 0, off_maps = 0, off_D = 0, table_used = 0;
  long long d_elems = 0;
  size_t workspace = 0;
  bool pinned = false;                      // host image from cudaHostAlloc
  bool dirty = true;                        // tables changed since the last upload
  const void* uploaded_ws = nullptr;
  int uploaded_dev = -1;
  // Side streams (device side_dev) on which the groups after the first run
  // concurrently with it: forked from the caller's stream after the queue
  // counters are reset, joined back before the call returns.
  static constexpr int kSide = 8;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSide] = {};
  int n_side = 0;
  int side_dev = -1;
  std::mutex mu;
};

namespace {

// MRC runs one lane per row (no sweep); L-MMSE and ZF may split a row over two lanes.
int lanes_per_row_default(int arch, int UP, int equalizer) {
  return (equalizer != FFEQ_MRC && equalizer != FFEQ_LAMA && arch == FFEQ_PD && UP == 16) ? 2 : 1;
}

bool lpr_allowed(int UP, int lpr, int equalizer) {
  return lpr == 1 || (lpr == 2 && UP <= 16 && equalizer != FFEQ_MRC && equalizer != FFEQ_LAMA);
}

// Smallest CTA width that holds the widest unit of the group.
int min_threads(const Group& g) { return ((g.max_ceff * g.UP * g.lpr + 31) / 32) * 32; }

bool threads_allowed(const Group& g, int threads, int lpr, int equalizer) {
  if (threads < 32 || threads > 512 || threads % 32 != 0) return false;
  const int slots = threads / (g.UP * lpr);   // UP * lpr divides 32
  if (slots < g.max_ceff || slots > ffeq::kTileSlots) return false;
  return ffeq::solve_batch_smem_bytes(g.UP, lpr, threads, equalizer) <= kSolveSmemLimit;
}

// Tile packing of one group into the table image (next fit over the solve order).
void build_tiles(ffeq_batch* b, Group& g, long long tile_first) {
  ffeq::SolveTile* tiles = reinterpret_cast<ffeq::SolveTile*>(b->host + b->off_tiles);
  unsigned short* maps = reinterpret_cast<unsigned short*>(b->host + b->off_maps);
  const int slots = g.threads / (g.UP * g.lpr);
  long long nt = 0;
  int used = slots;   // forces a new tile on the first unit
  for (long long q = 0; q < g.n_units; ++q) {
    const int ce = b->units[b->solve_order[g.first + q]].Ceff;
    if (used + ce > slots) {
      ffeq::SolveTile& t = tiles[tile_first + nt];
      t.first = static_cast<int>(q);
      t.count = 0;
      std::fill(maps + (tile_first + nt) * ffeq::kTileSlots, maps + (tile_first + nt + 1) * ffeq::kTileSlots,
                static_cast<unsigned short>(0xffff));
      ++nt;
      used = 0;
    }
    ffeq::SolveTile& t = tiles[tile_first + nt - 1];
    unsigned short* m = maps + (tile_first + nt - 1) * ffeq::kTileSlots;
    for (int c = 0; c < ce; ++c) m[used + c] = static_cast<unsigned short>((t.count << 8) | c);
    ++t.count;
    used += ce;
  }
  g.tile_first = tile_first;
  g.n_tiles = nt;
}

// Rebuild the descriptor and tile tables from the current tuning.
void build_tables(ffeq_batch* b) {
  ffeq::BatchDesc* gd = reinterpret_cast<ffeq::BatchDesc*>(b->host + b->off_gram);
  ffeq::BatchDesc* sd = reinterpret_cast<ffeq::BatchDesc*>(b->host + b->off_solve);
  std::memset(b->host, 0, b->off_gram);
  for (long long q = 0; q < b->n_units; ++q) {
    gd[q] = b->units[b->gram_order[q]];
    sd[q] = b->units[b->solve_order[q]];
  }
  long long tf = 0;
  for (Group& g : b->groups) {
    build_tiles(b, g, tf);
    tf += g.n_tiles;
  }
  b->table_used = b->off_maps + static_cast<size_t>(tf) * ffeq::kTileSlots * sizeof(unsigned short);
  b->dirty = true;
}

ffeq_status validate_instance(const ffeq_batch_config& cfg, const ffeq_instance& in) {
  if (in.B <= 0 || in.U <= 0 || in.C <= 0 || in.n_sc < 0 || in.n_sym <= 0) return FFEQ_ERR_INVALID_ARG;
  if (in.B % in.C != 0) return FFEQ_ERR_INVALID_ARG;
  if (!(in.N0 >= 0.f) || !std::isfinite(in.N0) || !(in.Es > 0.f) || !std::isfinite(in.Es))
    return FFEQ_ERR_INVALID_ARG;
  const bool lama = cfg.equalizer == FFEQ_LAMA;
  if (lama && !(in.N0 > 0.f)) return FFEQ_ERR_INVALID_ARG;   // the LAMA denoiser needs tau > 0
  if (in.U > 32 || in.n_sym > ffeq::kNsymMax) return FFEQ_ERR_UNSUPPORTED;
  const long long nsc = in.n_sc, U = in.U, B = in.B, NS = in.n_sym;
  const long long Ceff = cfg.arch == FFEQ_FD ? in.C : 1;
  auto in_range = [](long long off, long long n, long long extent) {
    return off >= 0 && n >= 0 && off <= extent && n <= extent - off;
  };
  if (!in_range(in.h_off, nsc * U * B, cfg.h_elems) || !in_range(in.y_off, nsc * NS * B, cfg.y_elems) ||
      !in_range(in.z_off, nsc * NS * U, cfg.z_elems) ||
      !in_range(in.sigma2_off, nsc * U * (lama ? NS : 1), cfg.sigma2_elems))   // LAMA: per received vector
    return FFEQ_ERR_INVALID_ARG;
  if (cfg.llr_bits && !in_range(in.llr_off, nsc * NS * U * cfg.llr_bits, cfg.llr_elems))
    return FFEQ_ERR_INVALID_ARG;
  if (cfg.info_elems > 0 && !in_range(in.info_off, nsc * Ceff, cfg.info_elems)) return FFEQ_ERR_INVALID_ARG;
  const int UP = ffeq::padded_users(in.U);
  if (Ceff > ffeq::kTileSlots || Ceff * UP > 512) return FFEQ_ERR_UNSUPPORTED;
  const ffeq::GramCaps gc =
      ffeq::gram_instance_caps(cfg.precision, in.B, in.U, in.n_sym, static_cast<int>(Ceff), ffeq::kGram16);
  if (ffeq::gram_stages_fit_bytes(gc.stage_elems, static_cast<size_t>(gc.slots) * gc.slot_elems * 8, false,
                                  ffeq::gram_smem_budget(ffeq::kGram16)) < 1)
    return FFEQ_ERR_UNSUPPORTED;
  return FFEQ_OK;
}

ffeq_status cuda_status(cudaError_t e) {
  return e == cudaSuccess ? FFEQ_OK : static_cast<ffeq_status>(ffeq::record_cuda_error(e));
}

}  // namespace

extern "C" {

ffeq_status ffeq_batch_create(ffeq_batch** out, const ffeq_batch_config* cfg, const ffeq_instance* inst,
                              int n_inst) {
  if (!out || !cfg || n_inst < 0 || (n_inst > 0 && !inst)) return FFEQ_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->arch != FFEQ_PD && cfg->arch != FFEQ_FD) return FFEQ_ERR_INVALID_ARG;
  if (cfg->precision != FFEQ_FP32 && cfg->precision != FFEQ_TF32X3 && cfg->precision != FFEQ_BF16X3 &&
      cfg->precision != FFEQ_FP16X3)
    return FFEQ_ERR_INVALID_ARG;
  if (cfg->estimate != FFEQ_UNBIASED && cfg->estimate != FFEQ_LITERAL) return FFEQ_ERR_INVALID_ARG;
  if (cfg->equalizer != FFEQ_LMMSE && cfg->equalizer != FFEQ_ZF && cfg->equalizer != FFEQ_MRC &&
      cfg->equalizer != FFEQ_LAMA)
    return FFEQ_ERR_INVALID_ARG;
  if (cfg->equalizer == FFEQ_LAMA ? (cfg->lama_iters < 1 || cfg->lama_iters > 64 || cfg->llr_bits == 0)
                                  : cfg->lama_iters != 0)
    return FFEQ_ERR_INVALID_ARG;   // LAMA's prior is the LLR constellation
  if (cfg->llr_bits != 0 && cfg->llr_bits != 2 && cfg->llr_bits != 4 && cfg->llr_bits != 6 && cfg->llr_bits != 8)
    return FFEQ_ERR_INVALID_ARG;
  if (cfg->h_elems < 0 || cfg->y_elems < 0 || cfg->z_elems < 0 || cfg->sigma2_elems < 0 || cfg->llr_elems < 0 ||
      cfg->info_elems < 0)
    return FFEQ_ERR_INVALID_ARG;
  for (int i = 0; i < n_inst; ++i) {
    const ffeq_status st = validate_instance(*cfg, inst[i]);
    if (st != FFEQ_OK) return st;
  }
  ffeq_batch* b = new (std::nothrow) ffeq_batch;
  if (!b) return FFEQ_ERR_INVALID_ARG;
  b->cfg = *cfg;
  b->n_inst = n_inst;

  // Units in instance order, with their workspace slices.
  std::vector<long long> inst_first(n_inst + 1, 0);
  long long d_off = 0;
  for (int i = 0; i < n_inst; ++i) {
    const ffeq_instance& in = inst[i];
    const int Ceff = cfg->arch == FFEQ_FD ? in.C : 1;
    inst_first[i] = static_cast<long long>(b->units.size());
    double scale = 0.0;
    if (cfg->llr_bits) {
      const double L = static_cast<double>(1 << (cfg->llr_bits / 2));
      scale = std::sqrt(static_cast<double>(in.Es) / (2.0 * (L * L - 1.0) / 3.0));
    }
    for (int k = 0; k < in.n_sc; ++k) {
      ffeq::BatchDesc d{};
      const long long U = in.U, B = in.B, NS = in.n_sym;
      d.h_off = in.h_off + k * U * B;
      d.y_off = in.y_off + k * NS * B;
      d.z_off = in.z_off + k * NS * U;
      d.s2_off = in.sigma2_off + k * U * (cfg->equalizer == FFEQ_LAMA ? NS : 1);
      d.llr_off = cfg->llr_bits ? in.llr_off + k * NS * U * cfg->llr_bits : 0;
      d.info_off = cfg->info_elems > 0 ? in.info_off + k * Ceff : 0;
      d.d_off = d_off;
      d_off += static_cast<long long>(Ceff) * (U + NS) * U;
      d_off += d_off & 1;   // every unit's slice 16-byte aligned (paired stores of the contraction)
      d.B = in.B;
      d.U = in.U;
      d.Ceff = Ceff;
      d.n_sym = in.n_sym;
      d.N0 = in.N0;
      // Zero forcing is the L-MMSE sweep with rho = 0 (and the literal pairs).
      d.rho = cfg->equalizer == FFEQ_ZF ? 0.f
                                         : static_cast<float>(static_cast<double>(in.N0) / static_cast<double>(in.Es));
      d.Es = in.Es;
      d.llr_scale = static_cast<float>(scale);
      d.inst = i;
      b->units.push_back(d);
    }
  }
  inst_first[n_inst] = static_cast<long long>(b->units.size());
  b->n_units = static_cast<long long>(b->units.size());
  b->d_elems = d_off;

  const size_t kBudget = ffeq::gram_smem_budget(ffeq::kGram16);
  // Groups: users padded to 8/16/32; within one, instances by decreasing
  // staged size, split where the combined shared-memory capacities stop fitting.
  for (int UP : {8, 16, 32}) {
    std::vector<int> ids;
    for (int i = 0; i < n_inst; ++i)
      if (ffeq::padded_users(inst[i].U) == UP && inst[i].n_sc > 0) ids.push_back(i);
    std::vector<int> st(n_inst), sl(n_inst), ns(n_inst);
    for (int i : ids) {
      const int Ceff = cfg->arch == FFEQ_FD ? inst[i].C : 1;
      const ffeq::GramCaps gc = ffeq::gram_instance_caps(cfg->precision, inst[i].B, inst[i].U, inst[i].n_sym, Ceff,
                                                         ffeq::kGram16);
      st[i] = gc.stage_elems;
      sl[i] = gc.slot_elems;
      ns[i] = gc.slots;
      // Slots are sized for the group's padded users (the kernel's slot stride).
      sl[i] = ((inst[i].U + inst[i].n_sym) * (UP + 1) + 1) & ~1;
    }
    // Instances without split-K partials first, then by decreasing staged size;
    // a group keeps the pipeline depth (up to 2) its first member allows alone.
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int c) {
      if ((ns[a] > 0) != (ns[c] > 0)) return ns[a] == 0;
      return st[a] > st[c];
    });
    size_t pos = 0;
    while (pos < ids.size()) {
      Group g{};
      g.UP = UP;
      g.bulk_ok = true;
      std::vector<int> members;
      int target = 1;
      for (; pos < ids.size(); ++pos) {
        const int i = ids[pos];
        const int cst = std::max(g.stage_elems, st[i]);
        const int csl = ns[i] > 0 ? std::max(g.slot_elems, sl[i]) : g.slot_elems;
        const int cns = std::max(g.n_slots, ns[i]);
        const int fit = ffeq::gram_stages_fit_bytes(cst, static_cast<size_t>(cns) * csl * 8, true, kBudget);
        if (members.empty()) target = std::min(2, fit);
        else if (fit < target) break;
        g.stage_elems = cst;
        g.slot_elems = csl;
        g.n_slots = cns;
        members.push_back(i);
        const int Ceff = cfg->arch == FFEQ_FD ? inst[i].C : 1;
        g.max_ceff = std::max(g.max_ceff, Ceff);
        if ((inst[i].B & 1) || (inst[i].h_off & 1) || (inst[i].y_off & 1)) g.bulk_ok = false;
      }
      g.max_stages = ffeq::gram_stages_fit_bytes(g.stage_elems, static_cast<size_t>(g.n_slots) * g.slot_elems * 8,
                                                 true, kBudget);
      g.first = static_cast<long long>(b->gram_order.size());
      std::vector<long long> us;
      for (int i : members)
        for (long long q = inst_first[i]; q < inst_first[i + 1]; ++q) us.push_back(q);
      g.n_units = static_cast<long long>(us.size());
      std::vector<long long> go = us, so = us;
      auto cost = [&](long long q) {
        const ffeq::BatchDesc& d = b->units[q];
        return static_cast<long long>(d.U + d.n_sym) * d.B;
      };
      std::stable_sort(go.begin(), go.end(), [&](long long a, long long c) { return cost(a) > cost(c); });
      std::stable_sort(so.begin(), so.end(),
                       [&](long long a, long long c) { return b->units[a].Ceff > b->units[c].Ceff; });
      b->gram_order.insert(b->gram_order.end(), go.begin(), go.end());
      b->solve_order.insert(b->solve_order.end(), so.begin(), so.end());
      g.stages = g.max_stages < 3 ? g.max_stages : 3;
      g.lpr = lanes_per_row_default(cfg->arch, UP, cfg->equalizer);
      g.threads = std::max(128, min_threads(g));
      if (!threads_allowed(g, g.threads, g.lpr, cfg->equalizer)) g.threads = min_threads(g);
      b->groups.push_back(g);
    }
  }
  if (b->groups.size() > static_cast<size_t>(kMaxGroups)) {
    delete b;
    return FFEQ_ERR_UNSUPPORTED;
  }

  // Table image: [queue counters][gram-order descriptors][solve-order descriptors][tiles][slot maps].
  const size_t nu = static_cast<size_t>(b->n_units);
  b->off_gram = kAlign;
  b->off_solve = align_up(b->off_gram + nu * sizeof(ffeq::BatchDesc));
  b->off_tiles = align_up(b->off_solve + nu * sizeof(ffeq::BatchDesc));
  b->off_maps = align_up(b->off_tiles + nu * sizeof(ffeq::SolveTile));
  b->off_D = align_up(b->off_maps + nu * ffeq::kTileSlots * sizeof(unsigned short));
  b->workspace = b->off_D + static_cast<size_t>(b->d_elems) * 8;
  void* host = nullptr;
  if (cudaHostAlloc(&host, b->off_D, cudaHostAllocDefault) != cudaSuccess) {
    (void)cudaGetLastError();   // no device here: keep a pageable image (uploads are then synchronous)
    host = nullptr;
  }
  if (!host) {
    host = new (std::nothrow) unsigned char[b->off_D];
    if (!host) {
      delete b;
      return FFEQ_ERR_INVALID_ARG;
    }
    b->host = static_cast<unsigned char*>(host);
    b->pinned = false;
  } else {
    b->host = static_cast<unsigned char*>(host);
    b->pinned = true;
  }
  build_tables(b);
  // Side streams for the groups after the first (none when there is one group,
  // or when no device is usable here: the groups then run in order).
  const int want = static_cast<int>(b->groups.size()) - 1 < ffeq_batch::kSide
                       ? static_cast<int>(b->groups.size()) - 1 : ffeq_batch::kSide;
  if (want > 0 && cudaGetDevice(&b->side_dev) == cudaSuccess &&
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess) {
    for (int j = 0; j < want; ++j) {
      if (cudaStreamCreateWithFlags(&b->side[j], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming) != cudaSuccess) {
        if (b->side[j]) cudaStreamDestroy(b->side[j]);
        b->side[j] = nullptr;
        break;
      }
      b->n_side = j + 1;
    }
  }
  (void)cudaGetLastError();
  *out = b;
  return FFEQ_OK;
}

void ffeq_batch_destroy(ffeq_batch* b) {
  if (!b) return;
  for (int j = 0; j < b->n_side; ++j) {
    cudaStreamDestroy(b->side[j]);
    cudaEventDestroy(b->join[j]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->pinned) {
    cudaFreeHost(b->host);
  } else {
    delete[] b->host;
  }
  delete b;
}

ffeq_status ffeq_batch_workspace_size(const ffeq_batch* b, size_t* bytes) {
  if (!b || !bytes) return FFEQ_ERR_INVALID_ARG;
  *bytes = b->workspace;
  return FFEQ_OK;
}

int ffeq_batch_groups(const ffeq_batch* b) { return b ? static_cast<int>(b->groups.size()) : 0; }

ffeq_status ffeq_batch_get_tuning(const ffeq_batch* b, int* values, int n) {
  if (!b || (n > 0 && !values) || n < 0) return FFEQ_ERR_INVALID_ARG;
  int w = 0;
  for (const Group& g : b->groups) {
    const int v[4] = {g.UP, g.stages, g.threads, g.lpr};
    for (int t = 0; t < 4 && w < n; ++t) values[w++] = v[t];
  }
  return FFEQ_OK;
}

ffeq_status ffeq_batch_set_tuning(ffeq_batch* b, const int* values, int n) {
  if (!b || n != 4 * static_cast<int>(b->groups.size()) || (n > 0 && !values)) return FFEQ_ERR_INVALID_ARG;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const Group& g = b->groups[gi];
    const int* v = values + 4 * gi;
    if (v[0] != g.UP || v[1] < 1 || v[1] > g.max_stages || !lpr_allowed(g.UP, v[3], b->cfg.equalizer))
      return FFEQ_ERR_INVALID_ARG;
    Group t = g;
    t.lpr = v[3];
    if (!threads_allowed(t, v[2], v[3], b->cfg.equalizer)) return FFEQ_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(b->mu);
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    Group& g = b->groups[gi];
    g.stages = values[4 * gi + 1];
    g.threads = values[4 * gi + 2];
    g.lpr = values[4 * gi + 3];
  }
  build_tables(b);
  return FFEQ_OK;
}

}  // extern "C"

namespace {

ffeq_status upload_locked(ffeq_batch* b, void* workspace, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemcpyAsync(static_cast<unsigned char*>(workspace) + b->off_gram, b->host + b->off_gram,
                      b->table_used - b->off_gram, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e);
  b->uploaded_ws = workspace;
  b->uploaded_dev = dev;
  b->dirty = false;
  return FFEQ_OK;
}

ffeq_status check_buffers(const ffeq_batch* b, const void* H, const void* y, const void* z, const float* sigma2,
                          const float* llr, const int* info, const void* workspace, size_t workspace_bytes) {
  if (!H || !y || !z || !sigma2 || !workspace) return FFEQ_ERR_INVALID_ARG;
  if (!aligned(H, 8) || !aligned(y, 8) || !aligned(z, 8) || !aligned(sigma2, 4)) return FFEQ_ERR_INVALID_ARG;
  if (b->cfg.llr_bits && (!llr || !aligned(llr, 4))) return FFEQ_ERR_INVALID_ARG;
  if (info && (b->cfg.info_elems <= 0 || !aligned(info, 4))) return FFEQ_ERR_INVALID_ARG;
  if (workspace_bytes < b->workspace || !aligned(workspace, kAlign)) return FFEQ_ERR_INVALID_ARG;
  return FFEQ_OK;
}

ffeq_status equalize_locked(ffeq_batch* b, const void* H, const void* y, void* z, float* sigma2, float* llr,
                            int* info, void* workspace, cudaStream_t st) {
  if (b->n_units == 0) return FFEQ_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (b->dirty || b->uploaded_ws != workspace || b->uploaded_dev != dev) {
    const ffeq_status s = upload_locked(b, workspace, st);
    if (s != FFEQ_OK) return s;
  }
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  e = cudaMemsetAsync(ws, 0, kAlign, st);   // work-queue counters
  if (e != cudaSuccess) return cuda_status(e);
  const bool bulk_ptrs = aligned(H, 16) && aligned(y, 16);
  ffeq::BatchLimits lim;
  lim.h = b->cfg.h_elems;
  lim.y = b->cfg.y_elems;
  lim.z = b->cfg.z_elems;
  lim.s2 = b->cfg.sigma2_elems;
  lim.llr = b->cfg.llr_bits ? b->cfg.llr_elems : 0;
  lim.info = b->cfg.info_elems;
  lim.d = b->d_elems;
  int* status = ffeq::device_status_ptr();
  const ffeq::BatchDesc* gdesc = reinterpret_cast<const ffeq::BatchDesc*>(ws + b->off_gram);
  const ffeq::BatchDesc* sdesc = reinterpret_cast<const ffeq::BatchDesc*>(ws + b->off_solve);
  const ffeq::SolveTile* tiles = reinterpret_cast<const ffeq::SolveTile*>(ws + b->off_tiles);
  const unsigned short* maps = reinterpret_cast<const unsigned short*>(ws + b->off_maps);
  float2* D = reinterpret_cast<float2*>(ws + b->off_D);
  // Group 0 on the caller's stream, the others on the side streams (round robin)
  // once they have waited for the counter reset; joined back at the end.
  const int n_side = dev == b->side_dev ? b->n_side : 0;
  if (n_side > 0 && (e = cudaEventRecord(b->fork, st)) != cudaSuccess) return cuda_status(e);
  bool used[ffeq_batch::kSide] = {};
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const Group& g = b->groups[gi];
    if (g.n_units == 0) continue;
    cudaStream_t gs = st;
    if (n_side > 0 && gi > 0) {
      const int j = static_cast<int>((gi - 1) % n_side);
      gs = b->side[j];
      if (!used[j]) {
        if ((e = cudaStreamWaitEvent(gs, b->fork, 0)) != cudaSuccess) return cuda_status(e);
        used[j] = true;
      }
    }
    ffeq::GramParams gp{};
    gp.H = static_cast<const float2*>(H);
    gp.y = static_cast<const float2*>(y);
    gp.D = D;
    gp.status = status;
    gp.U = g.UP;
    gp.bulk = g.bulk_ok && bulk_ptrs;
    gp.stages = gp.bulk ? g.stages : 1;
    gp.stage_elems = g.stage_elems;
    gp.slot_elems = g.slot_elems;
    gp.n_slots = g.n_slots;
    gp.n_units = static_cast<int>(g.n_units);
    gp.desc = gdesc + g.first;
    gp.queue = reinterpret_cast<int*>(ws) + gi;
    gp.UP = g.UP;
    gp.lim = lim;
    gp.variant = ffeq::kGram16;
    e = b->cfg.precision == FFEQ_FP32 ? ffeq::launch_gram_fp32(gp, gs)
                                      : ffeq::launch_gram_tc(gp, b->cfg.precision, gs);
    if (e != cudaSuccess) return cuda_status(e);
    ffeq::SolveParams sp{};
    sp.D = D;
    sp.z = static_cast<float2*>(z);
    sp.sigma2 = sigma2;
    sp.llr = b->cfg.llr_bits ? llr : nullptr;
    sp.info = info;
    sp.U = g.UP;
    sp.spc = 1;
    sp.unbiased = b->cfg.equalizer == FFEQ_LMMSE && b->cfg.estimate == FFEQ_UNBIASED;
    sp.equalizer = b->cfg.equalizer;
    sp.llr_bits = b->cfg.llr_bits;
    sp.desc = sdesc + g.first;
    sp.tiles = tiles + g.tile_first;
    sp.slot_map = maps + g.tile_first * ffeq::kTileSlots;
    sp.n_tiles = static_cast<int>(g.n_tiles);
    sp.n_desc = static_cast<int>(g.n_units);
    sp.threads = g.threads;
    sp.lim = lim;
    sp.status = status;
    if (b->cfg.equalizer == FFEQ_LAMA) {
      // One CTA per unit in contraction order, its received vectors a few at a time.
      sp.desc = gdesc + g.first;
      sp.lama_iters = b->cfg.lama_iters;
      const int lanes = ((g.max_ceff * g.UP + 31) / 32) * 32;
      sp.threads = lanes > 256 ? lanes : 256;
      e = ffeq::launch_lama_batch(sp, gs);
    } else {
      e = ffeq::launch_solve_batch(sp, g.lpr, gs);
    }
    if (e != cudaSuccess) return cuda_status(e);
  }
  for (int j = 0; j < n_side; ++j) {
    if (!used[j]) continue;
    if ((e = cudaEventRecord(b->join[j], b->side[j])) != cudaSuccess) return cuda_status(e);
    if ((e = cudaStreamWaitEvent(st, b->join[j], 0)) != cudaSuccess) return cuda_status(e);
  }
  return FFEQ_OK;
}

}  // namespace

extern "C" {

ffeq_status ffeq_batch_upload(ffeq_batch* b, void* workspace, size_t workspace_bytes, void* stream) {
  if (!b || !workspace || workspace_bytes < b->workspace || !aligned(workspace, kAlign)) return FFEQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(b->mu);
  if (b->n_units == 0) return FFEQ_OK;
  return upload_locked(b, workspace, static_cast<cudaStream_t>(stream));
}

ffeq_status ffeq_batch_equalize(ffeq_batch* b, const void* H, const void* y, void* z, float* sigma2, float* llr,
                                int* info, void* workspace, size_t workspace_bytes, void* stream) {
  if (!b) return FFEQ_ERR_INVALID_ARG;
  if (b->n_units == 0) return FFEQ_OK;
  const ffeq_status s = check_buffers(b, H, y, z, sigma2, llr, info, workspace, workspace_bytes);
  if (s != FFEQ_OK) return s;
  std::lock_guard<std::mutex> lock(b->mu);
  return equalize_locked(b, H, y, z, sigma2, llr, info, workspace, static_cast<cudaStream_t>(stream));
}

ffeq_status ffeq_batch_autotune(ffeq_batch* b, const void* H, const void* y, void* z, float* sigma2, float* llr,
                                int* info, void* workspace, size_t workspace_bytes, void* stream, int reps) {
  if (!b || reps < 1) return FFEQ_ERR_INVALID_ARG;
  if (b->n_units == 0) return FFEQ_OK;
  ffeq_status s = check_buffers(b, H, y, z, sigma2, llr, info, workspace, workspace_bytes);
  if (s != FFEQ_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return cuda_status(e);
  if (cap != cudaStreamCaptureStatusNone) return FFEQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(b->mu);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_status(e);
  }
  // Mean time of `reps` calls after one untimed call (which uploads changed tables).
  auto measure = [&](float& ms) -> ffeq_status {
    ffeq_status r = equalize_locked(b, H, y, z, sigma2, llr, info, workspace, st);
    if (r != FFEQ_OK) return r;
    cudaError_t ce = cudaEventRecord(e0, st);
    for (int i = 0; i < reps && ce == cudaSuccess; ++i) {
      r = equalize_locked(b, H, y, z, sigma2, llr, info, workspace, st);
      if (r != FFEQ_OK) return r;
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    return cuda_status(ce);
  };
  float best = 0.f;
  s = measure(best);
  for (size_t gi = 0; s == FFEQ_OK && gi < b->groups.size(); ++gi) {
    Group& g = b->groups[gi];
    // Contraction pipeline depth.
    for (int stg = 1; s == FFEQ_OK && stg <= g.max_stages && stg <= 3; ++stg) {
      if (stg == g.stages) continue;
      const int old = g.stages;
      g.stages = stg;
      float t = 0.f;
      s = measure(t);
      if (s == FFEQ_OK && t < best) best = t;
      else g.stages = old;
    }
    // Lanes per row and solve CTA width (tiles are rebuilt for each); LAMA
    // sizes its CTAs by the group's units instead.
    for (int lpr = 1; s == FFEQ_OK && lpr <= 2 && b->cfg.equalizer != FFEQ_LAMA; ++lpr) {
      if (!lpr_allowed(g.UP, lpr, b->cfg.equalizer)) continue;
      for (int th : {64, 128, 256, 512}) {
        if (s != FFEQ_OK) break;
        Group cand = g;
        cand.lpr = lpr;
        if ((lpr == g.lpr && th == g.threads) || !threads_allowed(cand, th, lpr, b->cfg.equalizer)) continue;
        const int old_l = g.lpr, old_t = g.threads;
        g.lpr = lpr;
        g.threads = th;
        build_tables(b);
        float t = 0.f;
        s = measure(t);
        if (s == FFEQ_OK && t < best) {
          best = t;
        } else {
          g.lpr = old_l;
          g.threads = old_t;
          build_tables(b);
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

}  // extern "C"
