// Host runtime of the CEM library: the C ABI declared in include/cem.h.
//
// cem_mesh_create builds the integer topology of the input mesh on the host
// (node incidence, edges in ascending (i, j) order, element -> edge map, edge
// fans, face adjacency), uploads it with the traction load, computes element
// geometry on the device and applies the notch splits with the run-time split
// path.  cem_step queues the five step kernels per step and, while crack-front
// elements exist, the energy-release-rate kernel plus (on steps with splits)
// the split sequence.
#include "cem_common.cuh"

#include <nvtx3/nvToolsExt.h>   // header-only; ranges cost nothing unless a profiler is attached

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

static thread_local std::string g_create_error;

int cem_fail(cem_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cem_cuda_fail(cem_ctx* c, cudaError_t e, const char* what) {
    return cem_fail(c, CEM_ECUDA, std::string("CUDA error '") + cudaGetErrorString(e) + "' in " + what);
}

int64_t cem_reduction_doubles();

void* cem_dalloc_bytes(cem_ctx* c, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    void* q = nullptr;
    if (c->alloc) {
        q = c->alloc(bytes, (void*)c->stream, c->alloc_user);
    } else if (cudaMalloc(&q, bytes) != cudaSuccess) {
        q = nullptr;
    }
    if (!q) return nullptr;
    c->allocs.push_back(q);
    c->bytes += (int64_t)bytes;
    return q;
}

namespace {

const int LE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

template <class T>
bool dalloc(cem_ctx* c, T*& p, int64_t n) {
    p = (T*)cem_dalloc_bytes(c, (size_t)std::max<int64_t>(n, 1) * sizeof(T));
    return p != nullptr;
}

int select_device(cem_ctx* c) {
    CEM_CK(c, cudaSetDevice(c->device));
    return CEM_OK;
}

template <class T>
int upload(cem_ctx* c, T* dst, const T* src, int64_t n) {
    if (n <= 0) return CEM_OK;
    CEM_CK(c, cudaMemcpyAsync(dst, src, (size_t)n * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return CEM_OK;
}

int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// [0, n) split into nt contiguous chunks of `size` items (the last one shorter or empty),
// one per host core (one chunk below 16,384 items).
struct Chunks {
    int64_t nt, size;
};
Chunks chunks_of(int64_t n) {
    int64_t nt = std::max<int64_t>(1, std::min<int64_t>(std::thread::hardware_concurrency(), 64));
    if (n < 16384) nt = 1;
    return {nt, std::max<int64_t>(1, (n + nt - 1) / nt)};
}

// f(k, begin, end) for chunk k of chunks_of(n), the chunks on the host's cores.  Every
// caller writes disjoint output slots (or per-chunk buffers), so the result does not
// depend on the split.
template <class F>
void parallel_chunks(int64_t n, F f) {
    const Chunks ch = chunks_of(n);
    if (ch.nt == 1) {
        f((int64_t)0, (int64_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    for (int64_t k = 0; k < ch.nt; ++k) {
        const int64_t a = std::min(n, k * ch.size), b = std::min(n, a + ch.size);
        th.emplace_back(f, k, a, b);
    }
    for (auto& t : th) t.join();
}

template <class F>
void parallel_for(int64_t n, F f) {
    parallel_chunks(n, [&](int64_t, int64_t a, int64_t b) { f(a, b); });
}

struct HostTopo {
    std::vector<int> inc_off, inc;          // node -> element*4+local, ascending
    std::vector<int> e_off, e_nbr;          // node i -> sorted neighbours j > i (edge ids e_off[i] + r)
    std::vector<int> t2e;                   // [6][T0]
    std::vector<int> fan_off, fan;          // edge -> elements, ascending
    std::vector<int> face_nbr;              // [4][T0]
};

int build_topology(cem_ctx* c, const std::vector<int>& conn, HostTopo& H) {
    const int64_t N = c->N0, T = c->T0;
    // node -> element * 4 + local, ascending: a counting sort by node.  Each chunk of
    // consecutive entries q = 4 element + local counts its entries per node; a node's list
    // then takes chunk 0's entries, chunk 1's, ..., each in ascending q, so the lists come
    // out ascending without a sort or an atomic.
    H.inc_off.assign(N + 1, 0);
    {
        const Chunks ch = chunks_of(4 * T);
        // per chunk: count per node, then its first slot (each chunk clears its own row)
        std::unique_ptr<int[]> pos(new int[(size_t)ch.nt * N]);
        parallel_chunks(4 * T, [&](int64_t k, int64_t a, int64_t b) {
            int* p = pos.get() + k * N;
            std::fill(p, p + N, 0);
            for (int64_t q = a; q < b; ++q) ++p[conn[q]];
        });
        parallel_for(N, [&](int64_t a, int64_t b) {
            for (int64_t i = a; i < b; ++i) {
                int s = 0;
                for (int64_t k = 0; k < ch.nt; ++k) s += pos[k * N + i];
                H.inc_off[i + 1] = s;
            }
        });
        for (int64_t i = 0; i < N; ++i) H.inc_off[i + 1] += H.inc_off[i];
        parallel_for(N, [&](int64_t a, int64_t b) {
            for (int64_t i = a; i < b; ++i) {
                int run = H.inc_off[i];
                for (int64_t k = 0; k < ch.nt; ++k) {
                    const int cnt = pos[k * N + i];
                    pos[k * N + i] = run;
                    run += cnt;
                }
            }
        });
        H.inc.assign(4 * T, 0);
        parallel_chunks(4 * T, [&](int64_t k, int64_t a, int64_t b) {
            int* p = pos.get() + k * N;
            for (int64_t q = a; q < b; ++q) H.inc[p[conn[q]]++] = (int)q;
        });
    }
    // edges: for each node the sorted distinct neighbours with larger id (counted, then
    // written, node by node on all host cores)
    auto neighbours = [&](int64_t i, std::vector<int>& buf) {
        buf.clear();
        for (int q = H.inc_off[i]; q < H.inc_off[i + 1]; ++q) {
            const int t = H.inc[q] >> 2;
            for (int l = 0; l < 4; ++l) {
                const int j = conn[(int64_t)t * 4 + l];
                if (j > i) buf.push_back(j);
            }
        }
        std::sort(buf.begin(), buf.end());
        buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    };
    // each chunk of nodes keeps its lists in a buffer of its own, copied into place once
    // the offsets are known
    H.e_off.assign(N + 1, 0);
    {
        std::vector<std::vector<int>> part(chunks_of(N).nt);
        parallel_chunks(N, [&](int64_t k, int64_t a, int64_t b) {
            std::vector<int> buf;
            for (int64_t i = a; i < b; ++i) {
                neighbours(i, buf);
                H.e_off[i + 1] = (int)buf.size();
                part[k].insert(part[k].end(), buf.begin(), buf.end());
            }
        });
        for (int64_t i = 0; i < N; ++i) H.e_off[i + 1] += H.e_off[i];
        H.e_nbr.assign(H.e_off[N], 0);
        parallel_chunks(N, [&](int64_t k, int64_t a, int64_t b) {
            if (a < b) std::copy(part[k].begin(), part[k].end(), H.e_nbr.begin() + H.e_off[a]);
        });
    }
    c->E0 = (int64_t)H.e_nbr.size();
    c->max_inc0 = 0;
    for (int64_t i = 0; i < N; ++i) c->max_inc0 = std::max<int64_t>(c->max_inc0, H.inc_off[i + 1] - H.inc_off[i]);
    H.t2e.assign(6 * T, 0);
    parallel_for(T, [&](int64_t a, int64_t b) {
        for (int64_t t = a; t < b; ++t)
            for (int l = 0; l < 6; ++l) {
                int x = conn[t * 4 + LE[l][0]], y = conn[t * 4 + LE[l][1]];
                if (x > y) std::swap(x, y);
                auto lo = H.e_nbr.begin() + H.e_off[x], hi = H.e_nbr.begin() + H.e_off[x + 1];
                auto it = std::lower_bound(lo, hi, y);
                H.t2e[l * T + t] = H.e_off[x] + (int)(it - lo);
            }
    });
    // fans: elements of each edge in ascending element order, the intersection of its
    // end nodes' (ascending) incidence lists; counted, then written, node by node
    auto fan_of = [&](int64_t x, int y, int* out) {   // writes when out != nullptr; returns the size
        int p = H.inc_off[x], pe = H.inc_off[x + 1], q = H.inc_off[y], qe = H.inc_off[y + 1], k = 0;
        while (p < pe && q < qe) {
            const int ta = H.inc[p] >> 2, tb = H.inc[q] >> 2;
            if (ta < tb) ++p;
            else if (tb < ta) ++q;
            else {
                if (out) out[k] = ta;
                ++k, ++p, ++q;
            }
        }
        return k;
    };
    // one intersection per edge, into per-chunk buffers copied into place afterwards
    H.fan_off.assign(c->E0 + 1, 0);
    {
        const Chunks ch = chunks_of(N);
        std::vector<std::vector<int>> part(ch.nt);
        std::vector<int64_t> pmax(ch.nt, 0);
        parallel_chunks(N, [&](int64_t k, int64_t a, int64_t b) {
            std::vector<int>& out = part[k];
            size_t used = 0;
            for (int64_t x = a; x < b; ++x)
                for (int e = H.e_off[x]; e < H.e_off[x + 1]; ++e) {
                    const int y = H.e_nbr[e];
                    // room for the shorter of the two lists (the buffer grows geometrically)
                    const size_t room = used + std::min(H.inc_off[x + 1] - H.inc_off[x], H.inc_off[y + 1] - H.inc_off[y]);
                    if (out.size() < room) out.resize(std::max(room, 2 * out.size()));
                    const int f = fan_of(x, y, out.data() + used);
                    used += f;
                    H.fan_off[e + 1] = f;
                    pmax[k] = std::max<int64_t>(pmax[k], f);
                }
            out.resize(used);
        });
        c->max_fan0 = *std::max_element(pmax.begin(), pmax.end());
        for (int64_t e = 0; e < c->E0; ++e) H.fan_off[e + 1] += H.fan_off[e];
        H.fan.assign(H.fan_off[c->E0], 0);
        parallel_chunks(N, [&](int64_t k, int64_t a, int64_t b) {
            if (a < b) std::copy(part[k].begin(), part[k].end(), H.fan.begin() + H.fan_off[H.e_off[a]]);
        });
    }
    // face adjacency (local face f is opposite local node f)
    H.face_nbr.assign(4 * T, -1);
    std::atomic<bool> non_manifold{false};
    // the element across face f (opposite local node f) shares the face's edge between its
    // first two nodes, so it is in that edge's fan: look for the fan element that also holds
    // the face's third node
    parallel_for(T, [&](int64_t a, int64_t b) {
        for (int64_t t = a; t < b; ++t)
            for (int f = 0; f < 4; ++f) {
                int fl[3], k = 0;
                for (int l = 0; l < 4; ++l)
                    if (l != f) fl[k++] = l;
                int le = 0;
                for (int l = 0; l < 6; ++l)
                    if ((LE[l][0] == fl[0] && LE[l][1] == fl[1]) || (LE[l][0] == fl[1] && LE[l][1] == fl[0])) le = l;
                const int e = H.t2e[le * T + t];
                const int third = conn[t * 4 + fl[2]];
                int found = -1, nfound = 0;
                for (int q = H.fan_off[e]; q < H.fan_off[e + 1]; ++q) {
                    const int s = H.fan[q];
                    if (s == t) continue;
                    bool has = false;
                    for (int l = 0; l < 4; ++l) has = has || conn[(int64_t)s * 4 + l] == third;
                    if (has) {
                        found = s;
                        ++nfound;
                    }
                }
                if (nfound > 1) non_manifold.store(true);
                H.face_nbr[f * T + t] = found;
            }
    });
    if (non_manifold.load())
        return cem_fail(c, CEM_EINVAL, "non-manifold mesh: a face is shared by more than two elements");
    return CEM_OK;
}

int sync_counts(cem_ctx* c) {
    CEM_CK(c, cudaMemcpyAsync(c->hcount, c->dcount, CNT_COUNT * sizeof(long long), cudaMemcpyDeviceToHost,
                              c->stream));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    return CEM_OK;
}

// Traction load on the host: triangles give t A / 3 to each node (Eq. 12);
// bilinear quadrilaterals give t * int N_a dA (2x2 Gauss).  Faces in order.
int traction_loads(cem_ctx* c, const cem_mesh_desc* d, int64_t N0, std::vector<double>& f) {
    const int nf = d->tface_nodes == 4 ? 4 : 3;
    f.assign(3 * N0, 0.0);
    const double g = 1.0 / std::sqrt(3.0);
    for (int64_t q = 0; q < d->n_tfaces; ++q) {
        const int* fn = d->tfaces + (int64_t)nf * q;
        for (int k = 0; k < nf; ++k)
            if (fn[k] < 0 || fn[k] >= N0) return cem_fail(c, CEM_EINVAL, "traction face node id out of range");
        const double* t = d->tvec + 3 * q;
        if (nf == 3) {
            const double* P = d->X + 3 * fn[0];
            const double* Q = d->X + 3 * fn[1];
            const double* R = d->X + 3 * fn[2];
            const double a[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
            const double b[3] = {R[0] - P[0], R[1] - P[1], R[2] - P[2]};
            const double cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
            const double A = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            for (int k = 0; k < 3; ++k)
                for (int r = 0; r < 3; ++r) f[k * N0 + fn[r]] += t[k] * A / 3.0;
        } else {
            const double sa[4] = {-1, 1, 1, -1}, ea[4] = {-1, -1, 1, 1};
            double w[4] = {0, 0, 0, 0};   // int N_a dA
            for (int gp = 0; gp < 4; ++gp) {
                const double s_ = (gp & 1) ? g : -g, r_ = (gp & 2) ? g : -g;
                double xs[3] = {0, 0, 0}, xr[3] = {0, 0, 0};
                for (int a = 0; a < 4; ++a)
                    for (int k = 0; k < 3; ++k) {
                        xs[k] += sa[a] * (1 + ea[a] * r_) / 4.0 * d->X[3 * fn[a] + k];
                        xr[k] += ea[a] * (1 + sa[a] * s_) / 4.0 * d->X[3 * fn[a] + k];
                    }
                const double cx = xs[1] * xr[2] - xs[2] * xr[1], cy = xs[2] * xr[0] - xs[0] * xr[2],
                             cz = xs[0] * xr[1] - xs[1] * xr[0];
                const double dA = std::sqrt(cx * cx + cy * cy + cz * cz);
                for (int a = 0; a < 4; ++a) w[a] += (1 + sa[a] * s_) * (1 + ea[a] * r_) / 4.0 * dA;
            }
            for (int k = 0; k < 3; ++k)
                for (int a = 0; a < 4; ++a) f[k * N0 + fn[a]] += t[k] * w[a];
        }
    }
    return CEM_OK;
}

// Hexahedral mesh (fixed topology): host topology from the 12 local edges,
// device arrays, geometry, load.  No notch, no splitting, one specimen.
const int HEX_LE[12][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6}, {6, 7}, {7, 4}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};

int create_hex_impl(const cem_mesh_desc* d, cem_ctx* c) {
    if (d->split_enabled || d->n_notch > 0)
        return cem_fail(c, CEM_EINVAL, "hexahedral meshes run with a fixed topology: split_enabled and n_notch must be 0");
    if (d->n_instances > 1) return cem_fail(c, CEM_EINVAL, "hexahedral meshes take one specimen");
    const int64_t N0 = d->n_nodes, T0 = d->n_tets;
    if (T0 >= (1ll << 26)) return cem_fail(c, CEM_EINVAL, "too many hexahedra for 32-bit entry ids");
    c->N0 = N0;
    c->T0 = T0;
    c->elem_type = CEM_ELEM_HEX8;
    c->npe = 8;
    c->epe = 12;
    c->split_enabled = 0;
    std::vector<int> conn(d->tets, d->tets + 8 * T0);
    const double g = 1.0 / std::sqrt(3.0);
    const double XI[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                             {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
    for (int64_t t = 0; t < T0; ++t) {
        const int* n = &conn[t * 8];
        for (int a = 0; a < 8; ++a) {
            if (n[a] < 0 || n[a] >= N0) return cem_fail(c, CEM_EINVAL, "element node id out of range");
            for (int b = a + 1; b < 8; ++b)
                if (n[a] == n[b]) return cem_fail(c, CEM_EINVAL, "element with a repeated node");
        }
        double V = 0.0;   // 2x2x2 Gauss of det J
        for (int q = 0; q < 8; ++q) {
            const double x = (q & 1) ? g : -g, y = (q & 2) ? g : -g, z = (q & 4) ? g : -g;
            double J[3][3] = {};
            for (int i = 0; i < 8; ++i) {
                const double a = XI[i][0], b = XI[i][1], cc = XI[i][2];
                const double gr[3] = {a * (1 + b * y) * (1 + cc * z) / 8, b * (1 + a * x) * (1 + cc * z) / 8,
                                      cc * (1 + a * x) * (1 + b * y) / 8};
                for (int r = 0; r < 3; ++r)
                    for (int k = 0; k < 3; ++k) J[r][k] += d->X[3 * n[i] + r] * gr[k];
            }
            V += J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        }
        if (!(V > 0.0) || !std::isfinite(V)) return cem_fail(c, CEM_EINVAL, "hexahedron without positive volume");
    }
    // topology: incidence (entries 8 t + l), edges from the 12 local edges, fans (entries 12 t + l)
    std::vector<int> inc_off(N0 + 1, 0), inc(8 * T0);
    for (int64_t t = 0; t < T0; ++t)
        for (int l = 0; l < 8; ++l) inc_off[conn[t * 8 + l] + 1]++;
    for (int64_t i = 0; i < N0; ++i) inc_off[i + 1] += inc_off[i];
    {
        std::vector<int> cur(inc_off.begin(), inc_off.end() - 1);
        for (int64_t t = 0; t < T0; ++t)
            for (int l = 0; l < 8; ++l) inc[cur[conn[t * 8 + l]]++] = (int)(t * 8 + l);
    }
    std::vector<std::pair<long long, int>> pk(12 * T0);   // (edge key, fan entry)
    for (int64_t t = 0; t < T0; ++t)
        for (int l = 0; l < 12; ++l) {
            long long x = conn[t * 8 + HEX_LE[l][0]], y = conn[t * 8 + HEX_LE[l][1]];
            if (x > y) std::swap(x, y);
            pk[t * 12 + l] = {x * N0 + y, (int)(t * 12 + l)};
        }
    std::sort(pk.begin(), pk.end());
    std::vector<int> t2e(12 * T0), fan(12 * T0), fan_off;
    int64_t E0 = 0;
    for (size_t q = 0; q < pk.size(); ++q) {
        if (q == 0 || pk[q].first != pk[q - 1].first) {
            fan_off.push_back((int)q);
            ++E0;
        }
        const int ent = pk[q].second;
        t2e[(ent % 12) * T0 + ent / 12] = (int)(E0 - 1);
        fan[q] = ent;
    }
    fan_off.push_back((int)pk.size());
    c->E0 = E0;
    c->max_inc0 = 0;
    for (int64_t i = 0; i < N0; ++i) c->max_inc0 = std::max<int64_t>(c->max_inc0, inc_off[i + 1] - inc_off[i]);
    c->max_fan0 = 0;
    for (int64_t e = 0; e < E0; ++e) c->max_fan0 = std::max<int64_t>(c->max_fan0, fan_off[e + 1] - fan_off[e]);
    std::vector<double> fload;
    if (int rc = traction_loads(c, d, N0, fload)) return rc;

    c->S_cap = 0;
    c->Tc = T0;
    c->Nc = N0;
    c->Ec = E0;
    c->fan_cap = 12 * T0;
    c->inc_cap = 8 * T0;
    if (int rc = select_device(c)) return rc;
    const int64_t Nc = c->Nc, Tc = c->Tc, Ec = c->Ec, HGV = cem_hex_geometry_values();
    const bool mixed = c->precision == CEM_MIXED;
    bool ok = true;
    ok = ok && dalloc(c, c->X, 3 * Nc) && dalloc(c, c->u, 3 * Nc) && dalloc(c, c->v, 3 * Nc) && dalloc(c, c->a, 3 * Nc);
    ok = ok && dalloc(c, c->fext, 3 * Nc) && dalloc(c, c->mass, Nc) && dalloc(c, c->minv, Nc);
    ok = ok && dalloc(c, c->inc_off, Nc) && dalloc(c, c->inc_cnt, Nc) && dalloc(c, c->inc_pool, c->inc_cap);
    ok = ok && dalloc(c, c->conn, 8 * Tc) && dalloc(c, c->t2e, 12 * Tc) && dalloc(c, c->anc, Tc);
    ok = ok && dalloc(c, c->active, Tc) && dalloc(c, c->Vg, HGV * Tc) && dalloc(c, c->vol, Tc);
    ok = ok && dalloc(c, c->lam, Tc) && dalloc(c, c->mu, Tc) && dalloc(c, c->Gc, Tc);
    if (mixed)
        ok = ok && dalloc(c, c->Vg32, HGV * Tc) && dalloc(c, c->h32, 8 * 12 * Tc) && dalloc(c, c->fp32, 32 * Tc) &&
             dalloc(c, c->uhl, 8 * Nc) && dalloc(c, c->cl32, Ec) && dalloc(c, c->cm32, Ec) && dalloc(c, c->sig32, 8 * Ec);
    else
        ok = ok && dalloc(c, c->h, 6 * 12 * Tc) && dalloc(c, c->fp, 24 * Tc) && dalloc(c, c->sig, 6 * Ec);
    ok = ok && dalloc(c, c->fan_off, Ec) && dalloc(c, c->fan_cnt, Ec) && dalloc(c, c->fan_pool, c->fan_cap);
    ok = ok && dalloc(c, c->cl, Ec) && dalloc(c, c->cm, Ec) && dalloc(c, c->sumV, Ec);
    ok = ok && dalloc(c, c->Ud, 1) && dalloc(c, c->dec_G, T0) && dalloc(c, c->ud_part, T0);
    ok = ok && dalloc(c, c->red_part, cem_reduction_doubles()) && dalloc(c, c->red_out, 8);
    ok = ok && dalloc(c, c->dcount, CNT_COUNT);
    if (c->n_dir > 0) ok = ok && dalloc(c, c->dir_key, c->n_dir) && dalloc(c, c->dir_v0, c->n_dir);
    if (!ok) return cem_fail(c, CEM_ENOMEM, "device allocation failed");
    CEM_CK(c, cudaMallocHost((void**)&c->hcount, CNT_COUNT * sizeof(long long)));
    CEM_CK(c, cudaMallocHost((void**)&c->hred, 8 * sizeof(double)));
    cudaStream_t s = c->stream;
    for (double* p : {c->u, c->v, c->a}) CEM_CK(c, cudaMemsetAsync(p, 0, 3 * Nc * sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->Ud, 0, sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->dcount, 0, CNT_COUNT * sizeof(long long), s));
    CEM_CK(c, cudaMemsetAsync(c->active, 1, Tc, s));
    if (mixed) CEM_CK(c, cudaMemsetAsync(c->uhl, 0, 8 * Nc * sizeof(float), s));
    {
        std::vector<double> Xs(3 * N0);
        for (int64_t i = 0; i < N0; ++i)
            for (int k = 0; k < 3; ++k) Xs[k * N0 + i] = d->X[3 * i + k];
        for (int k = 0; k < 3; ++k)
            if (int rc = upload(c, c->X + k * Nc, Xs.data() + k * N0, N0)) return rc;
        std::vector<int> cs(8 * T0);
        for (int64_t t = 0; t < T0; ++t)
            for (int l = 0; l < 8; ++l) cs[l * T0 + t] = conn[t * 8 + l];
        if (int rc = upload(c, c->conn, cs.data(), 8 * T0)) return rc;
        if (int rc = upload(c, c->t2e, t2e.data(), 12 * T0)) return rc;
        std::vector<int> anc(T0);
        std::iota(anc.begin(), anc.end(), 0);
        if (int rc = upload(c, c->anc, anc.data(), T0)) return rc;
        std::vector<int> fo(E0), fc(E0), io(N0), ic(N0);
        for (int64_t e = 0; e < E0; ++e) {
            fo[e] = fan_off[e];
            fc[e] = fan_off[e + 1] - fan_off[e];
        }
        for (int64_t i = 0; i < N0; ++i) {
            io[i] = inc_off[i];
            ic[i] = inc_off[i + 1] - inc_off[i];
        }
        if (int rc = upload(c, c->fan_off, fo.data(), E0)) return rc;
        if (int rc = upload(c, c->fan_cnt, fc.data(), E0)) return rc;
        if (int rc = upload(c, c->fan_pool, fan.data(), 12 * T0)) return rc;
        if (int rc = upload(c, c->inc_off, io.data(), N0)) return rc;
        if (int rc = upload(c, c->inc_cnt, ic.data(), N0)) return rc;
        if (int rc = upload(c, c->inc_pool, inc.data(), 8 * T0)) return rc;
        for (int k = 0; k < 3; ++k)
            if (int rc = upload(c, c->fext + k * Nc, fload.data() + k * N0, N0)) return rc;
        CEM_CK(c, cudaStreamSynchronize(s));
    }
    c->fan_top = 12 * T0;
    c->inc_top = 8 * T0;
    c->N = N0;
    c->T = T0;
    c->E = E0;
    c->n_active = T0;
    if (c->n_dir > 0) {
        if (int rc = upload(c, c->dir_key, c->h_dir_key.data(), c->n_dir)) return rc;
        if (int rc = upload(c, c->dir_v0, c->h_dir_v0.data(), c->n_dir)) return rc;
    }
    if (int rc = cem_hex_geometry(c, c->dec_G)) return rc;
    std::vector<double> hm(T0);
    CEM_CK(c, cudaMemcpyAsync(hm.data(), c->dec_G, T0 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CEM_CK(c, cudaStreamSynchronize(s));
    c->h_min = *std::min_element(hm.begin(), hm.end());
    c->inst_hmin.assign(1, c->h_min);
    return CEM_OK;
}

// Prescribed velocity components, keyed 4 * node + component (distinct), kept on the host until upload.
int parse_dirichlet(cem_ctx* c, const cem_mesh_desc* d) {
    const int64_t N0 = d->n_nodes;
    c->h_dir_key.assign(d->n_dirichlet, 0);
    c->h_dir_v0.assign(d->n_dirichlet, 0.0);
    for (int64_t q = 0; q < d->n_dirichlet; ++q) {
        const int i = d->dir_node[q], k = d->dir_comp[q];
        if (i < 0 || i >= N0 || k > 2) return cem_fail(c, CEM_EINVAL, "prescribed node or component out of range");
        if (!std::isfinite(d->dir_v0[q])) return cem_fail(c, CEM_EINVAL, "prescribed velocity must be finite");
        c->h_dir_key[q] = 4 * i + k;
        c->h_dir_v0[q] = d->dir_v0[q];
    }
    std::vector<int> sorted_keys(c->h_dir_key);
    std::sort(sorted_keys.begin(), sorted_keys.end());
    if (std::adjacent_find(sorted_keys.begin(), sorted_keys.end()) != sorted_keys.end())
        return cem_fail(c, CEM_EINVAL, "a node component is prescribed twice");
    c->n_dir = d->n_dirichlet;
    c->dir_t0 = d->dir_t0;
    return CEM_OK;
}

int create_impl(const cem_mesh_desc* d, cem_ctx* c) {
    if (!d || d->n_nodes <= 0 || d->n_tets <= 0 || !d->X || !d->tets)
        return cem_fail(c, CEM_EINVAL, "n_nodes, n_tets, X and tets are required");
    if (d->n_nodes >= (1ll << 30) || d->n_tets >= (1ll << 28))
        return cem_fail(c, CEM_EINVAL, "mesh too large for 32-bit ids");
    if (d->n_tfaces < 0 || (d->n_tfaces > 0 && (!d->tfaces || !d->tvec)))
        return cem_fail(c, CEM_EINVAL, "traction faces need tfaces and tvec");
    if (d->n_notch < 0 || (d->n_notch > 0 && (!d->notch_tet || !d->notch_side)))
        return cem_fail(c, CEM_EINVAL, "notch needs notch_tet and notch_side");
    if (d->precision != CEM_FP64 && d->precision != CEM_MIXED)
        return cem_fail(c, CEM_EINVAL, "precision must be CEM_FP64 or CEM_MIXED");
    if (d->split_mode != CEM_SPLIT_SUBDIVIDE && d->split_mode != CEM_SPLIT_DEACTIVATE)
        return cem_fail(c, CEM_EINVAL, "split_mode must be CEM_SPLIT_SUBDIVIDE or CEM_SPLIT_DEACTIVATE");
    if (d->g_variant != CEM_G_PRINCIPAL && d->g_variant != CEM_G_NORMAL)
        return cem_fail(c, CEM_EINVAL, "g_variant must be CEM_G_PRINCIPAL or CEM_G_NORMAL");
    if (d->n_dirichlet < 0 || (d->n_dirichlet > 0 && (!d->dir_node || !d->dir_comp || !d->dir_v0)))
        return cem_fail(c, CEM_EINVAL, "prescribed velocities need dir_node, dir_comp and dir_v0");
    if (!std::isfinite(d->dir_t0)) return cem_fail(c, CEM_EINVAL, "dir_t0 must be finite");
    c->device = d->device;
    c->stream = (cudaStream_t)d->stream;
    c->alloc = d->alloc;
    c->free_fn = d->free;
    c->alloc_user = d->alloc_user;
    c->dt_req = d->dt;
    c->cfl = d->cfl_factor > 0 ? d->cfl_factor : 0.5;
    c->split_enabled = d->split_enabled ? 1 : 0;
    c->split_mode = d->split_mode;
    c->g_variant = d->g_variant;
    c->precision = d->precision;
    for (int k = 0; k < TUNE_COUNT; ++k) c->tune[k] = cem_tune_default(k, c->precision);
    if (d->tface_nodes != 0 && d->tface_nodes != 3 && d->tface_nodes != 4)
        return cem_fail(c, CEM_EINVAL, "tface_nodes must be 3 or 4");
    if (int rc = parse_dirichlet(c, d)) return rc;
    if (d->elem_type == CEM_ELEM_HEX8) return create_hex_impl(d, c);
    if (d->elem_type != CEM_ELEM_TET4) return cem_fail(c, CEM_EINVAL, "elem_type must be CEM_ELEM_TET4 or CEM_ELEM_HEX8");

    const int64_t N0 = d->n_nodes, T0 = d->n_tets;
    c->N0 = N0;
    c->T0 = T0;
    std::vector<int> conn(d->tets, d->tets + 4 * T0);
    // node ids in range, no repeated node, non-zero finite volume; a negative signed
    // volume swaps local nodes 2 and 3 (element by element on all host cores)
    std::vector<char> swapped(T0, 0);
    std::atomic<int> bad{0};   // 1 id out of range, 2 repeated node, 3 zero volume
    parallel_for(T0, [&](int64_t a0, int64_t b0) {
        const double* X = d->X;
        for (int64_t t = a0; t < b0; ++t) {
            int* n = &conn[t * 4];
            bool ok = true;
            for (int a = 0; a < 4; ++a) ok = ok && n[a] >= 0 && n[a] < N0;
            if (!ok) {
                bad.store(1);
                continue;
            }
            for (int a = 0; a < 4; ++a)
                for (int b = a + 1; b < 4; ++b)
                    if (n[a] == n[b]) ok = false;
            if (!ok) {
                int z = 0;
                bad.compare_exchange_strong(z, 2);
                continue;
            }
            double e[3][3];
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 3; ++k) e[r][k] = X[3 * n[r + 1] + k] - X[3 * n[0] + k];
            const double V6 = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                              e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                              e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
            if (!(V6 != 0.0) || !std::isfinite(V6)) {
                int z = 0;
                bad.compare_exchange_strong(z, 3);
                continue;
            }
            if (V6 < 0) {
                std::swap(n[2], n[3]);
                swapped[t] = 1;
            }
        }
    });
    if (bad.load() == 1) return cem_fail(c, CEM_EINVAL, "element node id out of range");
    if (bad.load() == 2) return cem_fail(c, CEM_EINVAL, "element with a repeated node");
    if (bad.load() == 3) return cem_fail(c, CEM_EINVAL, "zero-volume element");
    // ensembles: element -> specimen map; every node must belong to one specimen
    std::vector<int> node_inst;
    c->n_inst = d->n_instances > 1 ? d->n_instances : 1;
    if (c->n_inst > 1) {
        if (!d->tet_instance) return cem_fail(c, CEM_EINVAL, "n_instances > 1 needs tet_instance");
        if (c->n_inst >= (1ll << 30)) return cem_fail(c, CEM_EINVAL, "too many instances");
        c->h_tet_inst.assign(d->tet_instance, d->tet_instance + T0);
        node_inst.assign(N0, -1);
        for (int64_t t = 0; t < T0; ++t) {
            const int i = c->h_tet_inst[t];
            if (i < 0 || i >= c->n_inst) return cem_fail(c, CEM_EINVAL, "tet_instance out of range");
            for (int l = 0; l < 4; ++l) {
                int& ni = node_inst[conn[t * 4 + l]];
                if (ni >= 0 && ni != i) return cem_fail(c, CEM_EINVAL, "a node is shared by two instances");
                ni = i;
            }
        }
        for (int64_t q = 0; q < N0; ++q)
            if (node_inst[q] < 0) node_inst[q] = 0;   // a node of no element: any specimen
    }
    HostTopo H;
    if (int rc = build_topology(c, conn, H)) return rc;
    const int64_t E0 = c->E0;

    // notch list: validated, oriented, side masks normalised (local node 0 on side 0), ascending
    std::vector<std::pair<int, int>> notch;
    for (int64_t q = 0; q < d->n_notch; ++q) {
        const int t = d->notch_tet[q];
        int m = d->notch_side[q] & 15;
        if (t < 0 || t >= T0) return cem_fail(c, CEM_EINVAL, "notch element id out of range");
        if (m == 0 || m == 15 || d->notch_side[q] > 15) return cem_fail(c, CEM_EINVAL, "notch side mask must cut the element");
        if (swapped[t]) m = (m & 3) | (((m >> 2) & 1) << 3) | (((m >> 3) & 1) << 2);
        if (m & 1) m = (~m) & 15;
        notch.push_back({t, m});
    }
    std::sort(notch.begin(), notch.end());
    for (size_t q = 1; q < notch.size(); ++q)
        if (notch[q].first == notch[q - 1].first) return cem_fail(c, CEM_EINVAL, "duplicate notch element");

    // capacities
    int64_t S_cap = d->split_capacity > 0 ? std::min<int64_t>(d->split_capacity, T0) : T0;
    if ((int64_t)notch.size() > S_cap) return cem_fail(c, CEM_EINVAL, "split_capacity below the notch size");
    if (!c->split_enabled) S_cap = (int64_t)notch.size();
    c->S_cap = S_cap;
    c->Tc = T0 + 6 * S_cap;
    c->Nc = N0 + std::min<int64_t>(2 * E0, 8 * S_cap);
    c->Ec = E0 + 22 * S_cap;
    c->fan_cap = 6 * c->Tc + (6 * T0) / 4 + 65536;
    c->inc_cap = 4 * c->Tc + T0 + 65536;
    c->hash_cap = next_pow2(std::max<int64_t>(1024, 2 * 22 * S_cap));
    const int64_t n_codes_cap = std::max<int64_t>(36 * S_cap, 1);
    const int64_t lim = (1ll << 31) - 1;
    if (c->Tc >= lim || c->Ec >= lim || c->Nc >= lim || c->fan_cap >= lim || c->inc_cap >= lim || 4 * c->Tc >= lim ||
        n_codes_cap >= lim)
        return cem_fail(c, CEM_EINVAL, "capacities exceed 32-bit indexing; lower split_capacity");
    const int64_t big = std::max({c->Ec, c->Nc, T0});
    const int64_t aff_cap = std::max(big, 42 * S_cap);   // affected marks of one split step: 7 S x 6
    const int64_t scan_max = std::max({2 * E0, c->Ec, c->Nc, T0, n_codes_cap, aff_cap});
    c->scan_blocks_cap = cem_scan_blocks_needed(scan_max);

    if (int rc = select_device(c)) return rc;
    const int64_t Nc = c->Nc, Tc = c->Tc, Ec = c->Ec;
    bool ok = true;
    ok = ok && dalloc(c, c->X, 3 * Nc) && dalloc(c, c->u, 3 * Nc) && dalloc(c, c->v, 3 * Nc) && dalloc(c, c->a, 3 * Nc);
    ok = ok && dalloc(c, c->fext, 3 * Nc) && dalloc(c, c->mass, Nc) && dalloc(c, c->minv, Nc);
    ok = ok && dalloc(c, c->inc_off, Nc) && dalloc(c, c->inc_cnt, Nc);
    ok = ok && dalloc(c, c->inc_pool, c->inc_cap) && dalloc(c, c->inc_pool2, c->inc_cap);
    ok = ok && dalloc(c, c->conn, 4 * Tc) && dalloc(c, c->t2e, 6 * Tc) && dalloc(c, c->anc, Tc);
    ok = ok && dalloc(c, c->active, Tc) && dalloc(c, c->Vg, 9 * Tc) && dalloc(c, c->vol, Tc);
    ok = ok && dalloc(c, c->lam, Tc) && dalloc(c, c->mu, Tc);
    const bool mixed = c->precision == CEM_MIXED;
    if (mixed)
        ok = ok && dalloc(c, c->Vg32, 9 * Tc) && dalloc(c, c->h32, 8 * Tc) && dalloc(c, c->fp32, 16 * Tc) &&
             dalloc(c, c->uhl, 8 * Nc) && dalloc(c, c->cl32, Ec) && dalloc(c, c->cm32, Ec) &&
             dalloc(c, c->sig32, 8 * Ec);
    else
        ok = ok && dalloc(c, c->h, 6 * Tc) && dalloc(c, c->fp, 12 * Tc) && dalloc(c, c->sig, 6 * Ec);
    ok = ok && dalloc(c, c->fan_off, Ec) && dalloc(c, c->fan_cnt, Ec);
    ok = ok && dalloc(c, c->fan_pool, c->fan_cap) && dalloc(c, c->fan_pool2, c->fan_cap);
    ok = ok && dalloc(c, c->cl, Ec) && dalloc(c, c->cm, Ec) && dalloc(c, c->sumV, Ec);
    ok = ok && dalloc(c, c->face_nbr, 4 * T0) && dalloc(c, c->side, T0) && dalloc(c, c->split_step, T0);
    ok = ok && dalloc(c, c->split_G, T0) && dalloc(c, c->Gc, T0) && dalloc(c, c->oe_n0, E0) && dalloc(c, c->oe_n1, E0);
    ok = ok && dalloc(c, c->node_of_key, 2 * E0) && dalloc(c, c->cand_flag, T0) && dalloc(c, c->cand_list, T0);
    ok = ok && dalloc(c, c->dec_mask, T0) && dalloc(c, c->dec_G, T0) && dalloc(c, c->split_list, T0);
    ok = ok && dalloc(c, c->act_orig, T0);
    ok = ok && dalloc(c, c->ext_of_int, Nc) && dalloc(c, c->int_of_ext, Nc) && dalloc(c, c->rn_map, Nc);
    if (ok) {   // renumbering scratch: the step's element-force and strain records are dead between steps
        int64_t kcap = 2048;
        while (kcap < Nc) kcap <<= 1;
        c->rn_keys_cap = kcap;
        const int64_t fp_bytes = (mixed ? 64 : 96) * Tc, h_bytes = (mixed ? 32 : 48) * Tc;
        if (fp_bytes >= 32 * Nc) c->rn_tmp = mixed ? (double*)c->fp32 : c->fp;
        else ok = dalloc(c, c->rn_tmp, 4 * Nc);
        if (h_bytes >= 8 * kcap) c->rn_keys = mixed ? (unsigned long long*)c->h32 : (unsigned long long*)c->h;
        else ok = ok && dalloc(c, c->rn_keys, kcap);
    }
    c->front_cap = std::min<int64_t>(T0, 1 << 16);
    const int64_t ff = 4 * c->front_cap;
    ok = ok && dalloc(c, c->ff_mask, ff) && dalloc(c, c->ff_prod, 4 * ff) && dalloc(c, c->ff_nrm, 6 * ff) &&
         dalloc(c, c->ff_edge, 3 * ff) && dalloc(c, c->ff_item, 3 * ff) && dalloc(c, c->ff_s, 3 * ff);
    ok = ok && dalloc(c, c->split_mask, T0) && dalloc(c, c->split_Gv, T0) && dalloc(c, c->ud_part, T0);
    ok = ok && dalloc(c, c->Ud, 1) && dalloc(c, c->ud_tet, T0);
    if (c->n_inst > 1)
        ok = ok && dalloc(c, c->node_inst, Nc) && dalloc(c, c->dtn, Nc) && dalloc(c, c->tet_inst, T0) &&
             dalloc(c, c->inst_dt_dev, c->n_inst);
    ok = ok && dalloc(c, c->hkeys, c->hash_cap) && dalloc(c, c->hvals, c->hash_cap) && dalloc(c, c->hfirst, c->hash_cap);
    ok = ok && dalloc(c, c->key_flag, 2 * E0) && dalloc(c, c->edge_flag, Ec) && dalloc(c, c->node_flag, Nc);
    ok = ok && dalloc(c, c->code_flag, n_codes_cap) && dalloc(c, c->new_keys, 2 * E0) && dalloc(c, c->sub_off, T0);
    ok = ok && dalloc(c, c->slot_of, n_codes_cap);
    ok = ok && dalloc(c, c->aff, aff_cap) && dalloc(c, c->aff_keep, aff_cap) && dalloc(c, c->aff_new, aff_cap) &&
         dalloc(c, c->aff_off, aff_cap);
    ok = ok && dalloc(c, c->add_cnt, big) && dalloc(c, c->cursor, big) && dalloc(c, c->scan_tmp, scan_max);
    const int64_t aff_cap_n = std::max(Nc, 28 * S_cap);   // node marks of one split step: 7 S x 4
    ok = ok && dalloc(c, c->aff_n, aff_cap_n) && dalloc(c, c->aff_keep_n, aff_cap_n) &&
         dalloc(c, c->aff_new_n, aff_cap_n) && dalloc(c, c->aff_off_n, aff_cap_n);
    ok = ok && dalloc(c, c->add_cnt_n, Nc) && dalloc(c, c->cursor_n, Nc);
    ok = ok && dalloc(c, c->scan_status, c->scan_blocks_cap) && dalloc(c, c->scan_ticket, 1);
    ok = ok && dalloc(c, c->red_part, cem_reduction_doubles()) && dalloc(c, c->red_out, 8);
    ok = ok && dalloc(c, c->dcount, CNT_COUNT);
    if (c->n_dir > 0) ok = ok && dalloc(c, c->dir_key, c->n_dir) && dalloc(c, c->dir_v0, c->n_dir);
    if (!ok) return cem_fail(c, CEM_ENOMEM, "device allocation failed");
    CEM_CK(c, cudaMallocHost((void**)&c->hcount, CNT_COUNT * sizeof(long long)));
    CEM_CK(c, cudaMallocHost((void**)&c->hred, 8 * sizeof(double)));

    cudaStream_t s = c->stream;
    // zero / sentinel initialisation
    CEM_CK(c, cudaMemsetAsync(c->u, 0, 3 * Nc * sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->v, 0, 3 * Nc * sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->a, 0, 3 * Nc * sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->fext, 0, 3 * Nc * sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->mass, 0, Nc * sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->minv, 0, Nc * sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->active, 0, Tc, s));
    CEM_CK(c, cudaMemsetAsync(c->lam, 0, Tc * sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->mu, 0, Tc * sizeof(double), s));
    if (mixed) {
        CEM_CK(c, cudaMemsetAsync(c->h32, 0, 8 * Tc * sizeof(float), s));
        CEM_CK(c, cudaMemsetAsync(c->fp32, 0, 16 * Tc * sizeof(float), s));
        CEM_CK(c, cudaMemsetAsync(c->sig32, 0, 8 * Ec * sizeof(float), s));
        CEM_CK(c, cudaMemsetAsync(c->uhl, 0, 8 * Nc * sizeof(float), s));
        CEM_CK(c, cudaMemsetAsync(c->cl32, 0, Ec * sizeof(float), s));
        CEM_CK(c, cudaMemsetAsync(c->cm32, 0, Ec * sizeof(float), s));
    } else {
        CEM_CK(c, cudaMemsetAsync(c->h, 0, 6 * Tc * sizeof(double), s));
        CEM_CK(c, cudaMemsetAsync(c->fp, 0, 12 * Tc * sizeof(double), s));
        CEM_CK(c, cudaMemsetAsync(c->sig, 0, 6 * Ec * sizeof(double), s));
    }
    CEM_CK(c, cudaMemsetAsync(c->side, 0, T0, s));
    CEM_CK(c, cudaMemsetAsync(c->split_step, 0, T0 * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->split_G, 0, T0 * sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->Gc, 0, T0 * sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->node_of_key, 0xFF, 2 * E0 * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->cand_flag, 0, T0, s));
    CEM_CK(c, cudaMemsetAsync(c->dec_mask, 0, T0, s));
    CEM_CK(c, cudaMemsetAsync(c->Ud, 0, sizeof(double), s));
    CEM_CK(c, cudaMemsetAsync(c->ud_tet, 0, T0 * sizeof(double), s));
    if (c->n_inst > 1) {
        CEM_CK(c, cudaMemsetAsync(c->dtn, 0, Nc * sizeof(double), s));
        if (int rc = upload(c, c->node_inst, node_inst.data(), N0)) return rc;
        if (int rc = upload(c, c->tet_inst, c->h_tet_inst.data(), T0)) return rc;
        CEM_CK(c, cudaStreamSynchronize(s));
    }
    CEM_CK(c, cudaMemsetAsync(c->hkeys, 0xFF, c->hash_cap * sizeof(unsigned long long), s));
    CEM_CK(c, cudaMemsetAsync(c->hvals, 0xFF, c->hash_cap * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->hfirst, 0x7F, c->hash_cap * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->key_flag, 0, 2 * E0, s));
    CEM_CK(c, cudaMemsetAsync(c->edge_flag, 0, Ec, s));
    CEM_CK(c, cudaMemsetAsync(c->node_flag, 0, Nc, s));
    CEM_CK(c, cudaMemsetAsync(c->code_flag, 0, n_codes_cap, s));
    CEM_CK(c, cudaMemsetAsync(c->add_cnt, 0, big * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->cursor, 0, big * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->add_cnt_n, 0, Nc * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->cursor_n, 0, Nc * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->fan_cnt, 0, Ec * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->fan_off, 0, Ec * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->inc_cnt, 0, Nc * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->inc_off, 0, Nc * sizeof(int), s));
    CEM_CK(c, cudaMemsetAsync(c->dcount, 0, CNT_COUNT * sizeof(long long), s));
    CEM_CK(c, cudaMemsetAsync(c->scan_status, 0, c->scan_blocks_cap * sizeof(unsigned long long), s));
    CEM_CK(c, cudaMemsetAsync(c->scan_ticket, 0, sizeof(unsigned int), s));
    if (int rc = cem_tma_init(c)) return rc;

    // uploads (structure of arrays)
    {
        std::vector<double> Xs(3 * N0);
        for (int64_t i = 0; i < N0; ++i)
            for (int k = 0; k < 3; ++k) Xs[k * N0 + i] = d->X[3 * i + k];
        for (int k = 0; k < 3; ++k)
            if (int rc = upload(c, c->X + k * Nc, Xs.data() + k * N0, N0)) return rc;
        if (int rc = cem_reorder_init(c, d->X, N0)) return rc;
        CEM_CK(c, cudaStreamSynchronize(s));
    }
    {
        std::vector<int> cs(4 * T0);
        for (int64_t t = 0; t < T0; ++t)
            for (int l = 0; l < 4; ++l) cs[l * T0 + t] = conn[t * 4 + l];
        for (int l = 0; l < 4; ++l)
            if (int rc = upload(c, c->conn + l * Tc, cs.data() + l * T0, T0)) return rc;
        for (int l = 0; l < 6; ++l)
            if (int rc = upload(c, c->t2e + l * Tc, H.t2e.data() + l * T0, T0)) return rc;
        std::vector<int> anc(T0);
        std::iota(anc.begin(), anc.end(), 0);
        if (int rc = upload(c, c->anc, anc.data(), T0)) return rc;
        CEM_CK(c, cudaMemsetAsync(c->active, 1, T0, s));
        if (int rc = upload(c, c->face_nbr, H.face_nbr.data(), 4 * T0)) return rc;
        CEM_CK(c, cudaStreamSynchronize(s));
    }
    {
        std::vector<int> fo(E0), fc(E0), n0(E0), n1(E0);
        for (int64_t e = 0; e < E0; ++e) {
            fo[e] = H.fan_off[e];
            fc[e] = H.fan_off[e + 1] - H.fan_off[e];
        }
        for (int64_t i = 0; i < N0; ++i)
            for (int q = H.e_off[i]; q < H.e_off[i + 1]; ++q) {
                n0[q] = (int)i;
                n1[q] = H.e_nbr[q];
            }
        if (int rc = upload(c, c->fan_off, fo.data(), E0)) return rc;
        if (int rc = upload(c, c->fan_cnt, fc.data(), E0)) return rc;
        if (int rc = upload(c, c->fan_pool, H.fan.data(), (int64_t)H.fan.size())) return rc;
        if (int rc = upload(c, c->oe_n0, n0.data(), E0)) return rc;
        if (int rc = upload(c, c->oe_n1, n1.data(), E0)) return rc;
        c->fan_top = (int64_t)H.fan.size();
        std::vector<int> io(N0), ic(N0);
        for (int64_t i = 0; i < N0; ++i) {
            io[i] = H.inc_off[i];
            ic[i] = H.inc_off[i + 1] - H.inc_off[i];
        }
        if (int rc = upload(c, c->inc_off, io.data(), N0)) return rc;
        if (int rc = upload(c, c->inc_cnt, ic.data(), N0)) return rc;
        if (int rc = upload(c, c->inc_pool, H.inc.data(), (int64_t)H.inc.size())) return rc;
        c->inc_top = (int64_t)H.inc.size();
        CEM_CK(c, cudaStreamSynchronize(s));
    }
    {   // traction load (Eq. 12)
        std::vector<double> f;
        if (int rc = traction_loads(c, d, N0, f)) return rc;
        for (int k = 0; k < 3; ++k)
            if (int rc = upload(c, c->fext + k * Nc, f.data() + k * N0, N0)) return rc;
        CEM_CK(c, cudaStreamSynchronize(s));
    }
    if (c->n_dir > 0) {
        if (int rc = upload(c, c->dir_key, c->h_dir_key.data(), c->n_dir)) return rc;
        if (int rc = upload(c, c->dir_v0, c->h_dir_v0.data(), c->n_dir)) return rc;
        CEM_CK(c, cudaStreamSynchronize(s));
    }
    c->N = N0;
    c->T = T0;
    c->E = E0;
    c->n_active = T0;

    // geometry of the input elements; h_min = min 3V / max face area
    if (int rc = cem_launch_geometry(c, 0, T0, c->dec_G)) return rc;
    if (c->n_inst == 1) {   // one specimen: the minimum on the device
        if (int rc = cem_device_min(c, c->dec_G, T0, &c->h_min)) return rc;
        c->inst_hmin.assign(1, c->h_min);
    } else {                // an ensemble: each specimen's minimum on the host
        std::vector<double> hm(T0);
        CEM_CK(c, cudaMemcpyAsync(hm.data(), c->dec_G, T0 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CEM_CK(c, cudaStreamSynchronize(s));
        c->h_min = *std::min_element(hm.begin(), hm.end());
        c->inst_hmin.assign(c->n_inst, 1e300);
        for (int64_t t = 0; t < T0; ++t) {
            const int i = c->h_tet_inst[t];
            c->inst_hmin[i] = std::min(c->inst_hmin[i], hm[t]);
        }
    }

    // notch: the run-time split path with no energy booked
    if (!notch.empty()) {
        const int64_t S = (int64_t)notch.size();
        std::vector<int> sl(S);
        std::vector<uint8_t> sm(S);
        std::vector<double> sg(S, 0.0);
        for (int64_t q = 0; q < S; ++q) {
            sl[q] = notch[q].first;
            sm[q] = (uint8_t)notch[q].second;
        }
        if (int rc = upload(c, c->split_list, sl.data(), S)) return rc;
        if (int rc = upload(c, c->split_mask, sm.data(), S)) return rc;
        if (int rc = upload(c, c->split_Gv, sg.data(), S)) return rc;
        if (int rc = cem_apply_splits(c, S, -1, 0)) return rc;
    }
    CEM_CK(c, cudaStreamSynchronize(s));
    return CEM_OK;
}

// ---- kernel timing: event pairs on the context's stream, resolved after a sync
cudaEvent_t ev_get(cem_ctx* c) {
    cudaEvent_t e = nullptr;
    if (!c->ev_pool.empty()) {
        e = c->ev_pool.back();
        c->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}

cudaEvent_t prof_begin(cem_ctx* c) {
    if (!c->prof_now) return nullptr;
    cudaEvent_t e = ev_get(c);
    if (e) cudaEventRecord(e, c->stream);
    return e;
}

void prof_end(cem_ctx* c, int id, cudaEvent_t a) {
    if (!a) return;
    cudaEvent_t b = ev_get(c);
    if (!b) return;
    cudaEventRecord(b, c->stream);
    c->ev_pending.push_back({id, a, b, c->step});
}

// Timing events of batch steps from `from` on (they returned at once) go back to the pool.
void prof_drop_from(cem_ctx* c, int64_t from) {
    size_t k = 0;
    for (auto& r : c->ev_pending) {
        if (r.step >= from) {
            c->ev_pool.push_back(r.a);
            c->ev_pool.push_back(r.b);
        } else {
            c->ev_pending[k++] = r;
        }
    }
    c->ev_pending.resize(k);
}

int prof_resolve(cem_ctx* c) {
    for (auto& r : c->ev_pending) {
        CEM_CK(c, cudaEventSynchronize(r.b));
        float ms = 0.f;
        CEM_CK(c, cudaEventElapsedTime(&ms, r.a, r.b));
        c->prof_ms[r.id] += ms;
        c->prof_n[r.id] += 1;
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->ev_pending.clear();
    return CEM_OK;
}

#define TIMED(c, id, expr)                 \
    do {                                   \
        cudaEvent_t ev_ = prof_begin(c);   \
        int rc_ = (expr);                  \
        prof_end(c, id, ev_);              \
        if (rc_) return rc_;               \
    } while (0)

// NVTX range for the duration of a scope (seen by nsys / ncu timelines)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// The front evaluation (Eqs. 16-18) on the side stream, forked from the context's
// stream after the edge stresses.  It reads the end-of-step displacement, the edge
// stresses and the crack topology.  FP64: u is already the end-of-step displacement
// and neither the force nor the node-update kernel writes u, the edge stresses or
// the topology (the FP64 node update writes v and a), so the evaluation runs beside
// both and joins before the split decision is read.  Mixed precision: the node update
// advances u, so the evaluation forms the end-of-step displacement from the stored
// u, v, a as the node update does (FrontU) and joins before the node update.
int make_side_stream(cem_ctx* c) {
    if (c->side_stream) return CEM_OK;
    // the highest priority: the block scheduler then starts the front's few blocks as
    // soon as an SM has room, ahead of the force kernel's blocks still waiting
    int lo = 0, hi = 0;
    CEM_CK(c, cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CEM_CK(c, cudaStreamCreateWithPriority(&c->side_stream, cudaStreamNonBlocking, hi));
    CEM_CK(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CEM_CK(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    return CEM_OK;
}

int launch_front_side(cem_ctx* c) {
    if (int rc = make_side_stream(c)) return rc;
    CEM_CK(c, cudaEventRecord(c->ev_fork, c->stream));
    CEM_CK(c, cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0));
    cudaStream_t main = c->stream;
    c->stream = c->side_stream;   // the front's launches and its timing events go to the side stream
    cudaEvent_t ev = prof_begin(c);
    int rc;
    {
        NvtxRange front("cem.front_G");
        rc = cem_launch_front_G(c, c->precision == CEM_MIXED ? 1 : 0);
    }
    prof_end(c, CEM_KERNEL_FRONT_G, ev);
    c->stream = main;
    if (rc) return rc;
    CEM_CK(c, cudaEventRecord(c->ev_join, c->side_stream));
    return CEM_OK;
}

// Launches one step; with crack-front elements the split decision is left on the
// device (CNT_SPLIT) for run_step or the end of a batch.
int launch_step(cem_ctx* c) {
    NvtxRange range("cem.step");
    if (c->tune_auto)
        if (int rc = cem_tune_maybe(c)) return rc;
    c->prof_now = c->prof && (c->step % c->prof_every == 0);
    // the front evaluation runs beside the force kernel (and, FP64, the node update)
    const bool fronts = c->split_enabled && c->n_cand > 0;
    const bool mix = c->precision == CEM_MIXED;
    if (!mix)   // mixed precision: the node update carries the predictor
        TIMED(c, CEM_KERNEL_PREDICT, cem_launch_predict(c));
    TIMED(c, CEM_KERNEL_STRAIN, cem_launch_strain(c));
    TIMED(c, CEM_KERNEL_EDGE_STRESS, cem_launch_edge_stress(c));
    if (fronts)
        if (int rc = launch_front_side(c)) return rc;
    TIMED(c, CEM_KERNEL_FORCE, cem_launch_force(c));
    if (fronts && mix) CEM_CK(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    TIMED(c, CEM_KERNEL_NODE_UPDATE, cem_launch_node_update(c, 0));
    if (int rc = cem_launch_prescribe(c, c->step + 1)) return rc;
    c->step += 1;
    if (fronts && !mix) CEM_CK(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    return CEM_OK;
}

// Applies the splits the front evaluation of the step just run decided (counters read).
int apply_step_splits(cem_ctx* c) {
    if (c->hcount[CNT_ERR] & DERR_SCAN_WAIT) return cem_fail(c, CEM_ETIMEOUT, "a scan's bounded look-back wait gave up");
    const int64_t S = c->hcount[CNT_SPLIT];
    if (S <= 0) return CEM_OK;
    if (c->n_split_all + S > c->S_cap)
        return cem_fail(c, CEM_ECAPACITY, "split capacity exhausted; splits of this step not applied");
    NvtxRange split("cem.split");
    int rc;
    // the splits, then a renumbering of node storage when the node count has grown enough
    TIMED(c, CEM_KERNEL_SPLIT, (rc = cem_apply_splits(c, S, c->step, 1)) ? rc : cem_reorder_maybe(c));
    return CEM_OK;
}

int run_step(cem_ctx* c, bool* split = nullptr) {
    const bool fronts = c->split_enabled && c->n_cand > 0;
    if (int rc = launch_step(c)) return rc;
    if (fronts) {
        if (int rc = sync_counts(c)) return rc;
        if (split) *split = c->hcount[CNT_SPLIT] > 0;
        if (int rc = apply_step_splits(c)) return rc;
    }
    if (c->ev_pending.size() > 4096) return prof_resolve(c);
    return CEM_OK;
}

// A batch: B steps launched back to back with crack-front elements, the split decision
// read once at the end.  Step r of the batch is gated (StepGate): when the front
// evaluation of step r decides splits, the kernels of steps r+1 .. B-1 return at once,
// and the host applies the splits after step r, as run_step would.  *ran = steps run.
int run_batch(cem_ctx* c, int64_t B, int64_t* ran, bool* split) {
    const int64_t step0 = c->step;
    CEM_CK(c, cudaMemsetAsync(c->dcount + CNT_HALT, 0, sizeof(long long), c->stream));
    int rc = CEM_OK;
    for (int64_t r = 0; r < B && rc == CEM_OK; ++r) {
        c->spec_r = r;
        rc = launch_step(c);
    }
    c->spec_r = -1;
    if (rc) return rc;
    if ((rc = sync_counts(c))) return rc;
    const int64_t h = c->hcount[CNT_HALT];
    *ran = h > 0 ? h : B;
    *split = h > 0;
    c->step = step0 + *ran;
    prof_drop_from(c, c->step);
    if (h > 0) {
        if ((rc = apply_step_splits(c))) return rc;
    } else if (c->hcount[CNT_ERR] & DERR_SCAN_WAIT) {
        return cem_fail(c, CEM_ETIMEOUT, "a scan's bounded look-back wait gave up");
    }
    if (c->ev_pending.size() > 4096) return prof_resolve(c);
    return CEM_OK;
}

// n steps: one at a time without crack-front elements (no host read between steps);
// with them, in batches whose length doubles after every batch without a split (up to
// spec_max) and falls back to 1 after a split.
int run_steps(cem_ctx* c, int64_t n) {
    for (int64_t q = 0; q < n;) {
        const bool fronts = c->split_enabled && c->n_cand > 0;
        const int64_t B = std::min(c->spec_len, n - q);
        int64_t ran = 1;
        bool split = false;
        if (fronts && B > 1) {
            if (int rc = run_batch(c, B, &ran, &split)) return rc;
        } else if (int rc = run_step(c, &split)) {
            return rc;
        }
        q += ran;
        if (fronts) {
            if (split) c->spec_len = 1;
            else if (B == c->spec_len) c->spec_len = std::min(2 * c->spec_len, c->spec_max);
        }
    }
    return CEM_OK;
}

}  // namespace

int cem_run_step(cem_ctx* c) { return run_step(c); }

// A TMA-gather wait of the edge stress that gave up (counters read): CEM_ETIMEOUT, flag cleared.
static int check_tma_wait(cem_ctx* c) {
    if (!(c->hcount[CNT_ERR] & DERR_TMA_WAIT)) return CEM_OK;
    CEM_CK(c, cudaMemsetAsync(c->dcount + CNT_ERR, 0, sizeof(long long), c->stream));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    return cem_fail(c, CEM_ETIMEOUT, "a bounded wait for the edge stress's TMA gathers gave up");
}

extern "C" {

int cem_mesh_create(const cem_mesh_desc* d, cem_ctx** out) {
    if (!out) return CEM_EINVAL;
    *out = nullptr;
    cem_ctx* c = new cem_ctx();
    int rc = create_impl(d, c);
    if (rc != CEM_OK) {
        g_create_error = c->err;
        cem_destroy(c);
        return rc;
    }
    *out = c;
    return CEM_OK;
}

int cem_set_material(cem_ctx* c, double rho, double nu, const double* E, int64_t nE, const double* Gc, int64_t nGc) {
    if (!c) return CEM_EINVAL;
    if (c->step > 0) return cem_fail(c, CEM_ESTATE, "material can only be set before the first step");
    if (!(rho > 0) || !(nu > -1.0 && nu < 0.5)) return cem_fail(c, CEM_EINVAL, "need rho > 0 and -1 < nu < 0.5");
    if (!E || !Gc || (nE != 1 && nE != c->T0) || (nGc != 1 && nGc != c->T0))
        return cem_fail(c, CEM_EINVAL, "E and Gc must have 1 or n_tets entries");
    double Emax = 0.0;
    for (int64_t q = 0; q < nE; ++q) {
        if (!(E[q] > 0) || !std::isfinite(E[q])) return cem_fail(c, CEM_EINVAL, "E must be positive");
        Emax = std::max(Emax, E[q]);
    }
    for (int64_t q = 0; q < nGc; ++q)
        if (!(Gc[q] >= 0) || !std::isfinite(Gc[q])) return cem_fail(c, CEM_EINVAL, "Gc must be non-negative");
    if (int rc = select_device(c)) return rc;
    c->rho = rho;
    c->nu = nu;
    // the T0-sized dec_G and ud_part buffers stage E and Gc
    if (int rc = upload(c, c->dec_G, E, nE)) return rc;
    if (int rc = upload(c, c->ud_part, Gc, nGc)) return rc;
    if (int rc = cem_launch_material(c, c->dec_G, (int)(nE == 1 ? 1 : 2), c->ud_part, (int)(nGc == 1 ? 1 : 2)))
        return rc;
    if (int rc = cem_launch_edge_coeffs(c, nullptr, 0)) return rc;
    if (int rc = cem_launch_node_mass(c, nullptr, 0)) return rc;
    // time step of every specimen: cfl * h_min / (2 c_d) at its largest modulus
    std::vector<double> Ei(c->n_inst, 0.0);
    for (int64_t t = 0; t < c->T0; ++t) {
        const int i = c->n_inst > 1 ? c->h_tet_inst[t] : 0;
        Ei[i] = std::max(Ei[i], nE == 1 ? E[0] : E[t]);
    }
    (void)Emax;
    c->inst_dt.assign(c->n_inst, 0.0);
    for (int64_t i = 0; i < c->n_inst; ++i) {
        const double lam = Ei[i] * nu / ((1 + nu) * (1 - 2 * nu)), mu = Ei[i] / (2 * (1 + nu));
        const double c_d = std::sqrt((lam + 2 * mu) / rho);
        c->inst_dt[i] = c->dt_req > 0 ? c->dt_req : c->cfl * c->inst_hmin[i] / (2.0 * c_d);
    }
    c->dt = *std::min_element(c->inst_dt.begin(), c->inst_dt.end());
    if (c->n_inst > 1) {
        if (int rc = upload(c, c->inst_dt_dev, c->inst_dt.data(), c->n_inst)) return rc;
        if (int rc = cem_launch_node_dt(c)) return rc;
    }
    // a_0 = M^-1 (f_ext - f_int(u_0))
    int rc;
    if ((rc = cem_launch_strain(c)) || (rc = cem_launch_edge_stress(c)) || (rc = cem_launch_force(c)) ||
        (rc = cem_launch_node_update(c, 1)) || (rc = cem_launch_prescribe(c, 0)))
        return rc;
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    c->material = true;
    return CEM_OK;
}

int cem_step(cem_ctx* c, int64_t n) {
    if (!c || n < 0) return CEM_EINVAL;
    if (!c->material) return cem_fail(c, CEM_ESTATE, "cem_set_material must be called before cem_step");
    if (int rc = select_device(c)) return rc;
    if (int rc = run_steps(c, n)) return rc;
    if (int rc = cem_launch_check_finite(c)) return rc;
    if (int rc = sync_counts(c)) return rc;
    if (int rc = check_tma_wait(c)) return rc;
    if (c->hcount[CNT_SCRATCH1]) return cem_fail(c, CEM_ENONFINITE, "non-finite displacement");
    return prof_resolve(c);
}

// n steps of a fixed-topology context in one persistent cooperative launch: the phases
// of each step are separated by grid barriers whose waits are bounded.
int cem_step_persistent(cem_ctx* c, int64_t n) {
    if (!c || n < 0) return CEM_EINVAL;
    if (!c->material) return cem_fail(c, CEM_ESTATE, "cem_set_material must be called before cem_step_persistent");
    if (c->elem_type != CEM_ELEM_TET4) return cem_fail(c, CEM_ESTATE, "the persistent step covers tetrahedral meshes");
    if (c->split_enabled && c->n_cand > 0)
        return cem_fail(c, CEM_ESTATE, "crack-front elements need the split test after every step: use cem_step");
    if (c->n_dir > 0)
        return cem_fail(c, CEM_ESTATE, "prescribed velocities are applied between steps: use cem_step");
    if (c->prof) return cem_fail(c, CEM_ESTATE, "kernel timing is on (cem_profile): use cem_step");
    if (int rc = select_device(c)) return rc;
    if (n == 0) return CEM_OK;
    if (c->tune_auto)   // the one-phase kernels' variants stay settled for the sizes
        if (int rc = cem_tune_maybe(c)) return rc;
    if (int rc = cem_launch_persistent(c, n)) return rc;
    if (int rc = sync_counts(c)) return rc;
    if (c->hcount[CNT_ERR] & DERR_BARRIER) {
        CEM_CK(c, cudaMemsetAsync(c->dcount + CNT_ERR, 0, sizeof(long long), c->stream));
        CEM_CK(c, cudaStreamSynchronize(c->stream));
        return cem_fail(c, CEM_ETIMEOUT,
                        "a grid barrier's bounded wait gave up; the steps of this call did not all run and the "
                        "state is not that of any step");
    }
    c->step += n;
    if (int rc = cem_launch_check_finite(c)) return rc;
    if (int rc = sync_counts(c)) return rc;
    if (c->hcount[CNT_SCRATCH1]) return cem_fail(c, CEM_ENONFINITE, "non-finite displacement");
    return CEM_OK;
}

int cem_set_step_batch(cem_ctx* c, int64_t max_steps) {
    if (!c) return CEM_EINVAL;
    if (max_steps < 1) return cem_fail(c, CEM_EINVAL, "max_steps must be at least 1");
    c->spec_max = max_steps;
    c->spec_len = std::min(c->spec_len, max_steps);
    return CEM_OK;
}

// n steps launched as one CUDA graph.  Without crack-front elements (splitting off, or
// none left) the topology cannot change over the steps.  With them the graph holds one
// batch of n gated steps (see run_batch): when the front evaluation of a step decides
// splits, the later steps of the graph return at once, the host applies the splits, and
// the rest of the call runs as cem_step runs it.  The graph is captured on a private
// stream the first time (or when n, the sizes, the topology or the launch variants
// change) and replayed on the context's stream; its kernels and arguments are those
// cem_step launches, so the results are bit-identical.
int cem_step_graph(cem_ctx* c, int64_t n) {
    if (!c || n < 0) return CEM_EINVAL;
    if (!c->material) return cem_fail(c, CEM_ESTATE, "cem_set_material must be called before cem_step_graph");
    if (c->n_dir > 0)
        return cem_fail(c, CEM_ESTATE, "prescribed velocities depend on the step number: use cem_step");
    if (c->prof) return cem_fail(c, CEM_ESTATE, "kernel timing is on (cem_profile): use cem_step");
    if (int rc = select_device(c)) return rc;
    if (n == 0) return CEM_OK;
    const bool fronts = c->split_enabled && c->n_cand > 0;
    // While the crack is active (the last step split, and no step since has run without a
    // split) a replay would end at its first step and the topology would change under every
    // capture: run as cem_step does until a step passes without a split.
    if (fronts && c->spec_len == 1 && c->n_split_run > 0) {
        if (int rc = run_steps(c, n)) return rc;
        if (int rc = cem_launch_check_finite(c)) return rc;
        if (int rc = sync_counts(c)) return rc;
        if (int rc = check_tma_wait(c)) return rc;
        if (c->hcount[CNT_SCRATCH1]) return cem_fail(c, CEM_ENONFINITE, "non-finite displacement");
        return CEM_OK;
    }
    if (c->tune_auto)   // settle the launch variants for the current sizes before capturing them
        if (int rc = cem_tune_maybe(c)) return rc;
    constexpr int K = cem_ctx::GRAPH_KEY;
    const int64_t key[K] = {n,      c->T,           c->E,       c->N,       c->n_cand,  c->n_act_orig,
                            fronts, c->topo_version, c->tune[0], c->tune[1], c->tune[2], c->tune[3]};
    if (!c->graph_exec || !std::equal(key, key + K, c->graph_key)) {
        if (c->graph_exec) {
            CEM_CK(c, cudaGraphExecDestroy(c->graph_exec));
            c->graph_exec = nullptr;
        }
        if (!c->cap_stream) CEM_CK(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        if (fronts)
            if (int rc = make_side_stream(c)) return rc;
        CEM_CK(c, cudaStreamSynchronize(c->stream));   // the state the graph starts from is in place
        const cudaStream_t main = c->stream;
        const int64_t step0 = c->step, launch0 = c->n_launch;
        c->stream = c->cap_stream;
        c->capturing = true;
        int rc = CEM_OK;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            if (fronts) e = cudaMemsetAsync(c->dcount + CNT_HALT, 0, sizeof(long long), c->cap_stream);
            for (int64_t q = 0; q < n && rc == CEM_OK && e == cudaSuccess; ++q) {
                c->spec_r = fronts ? q : -1;
                rc = launch_step(c);
            }
            c->spec_r = -1;
            const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
            if (e == cudaSuccess) e = e2;
        }
        c->stream = main;
        c->capturing = false;
        c->step = step0;   // capture launched nothing: the steps run at replay
        c->n_graph_launch = c->n_launch - launch0;
        c->n_launch = launch0;
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cem_cuda_fail(c, e, "stream capture of the step graph");
        }
        e = cudaGraphInstantiate(&c->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->graph_exec = nullptr;
            return cem_cuda_fail(c, e, "cudaGraphInstantiate");
        }
        std::copy(key, key + K, c->graph_key);
    }
    CEM_CK(c, cudaGraphLaunch(c->graph_exec, c->stream));
    cem_launched(c, (int)c->n_graph_launch);
    if (!fronts) {
        c->step += n;
    } else {
        if (int rc = sync_counts(c)) return rc;
        const int64_t h = c->hcount[CNT_HALT];
        const int64_t ran = h > 0 ? h : n;
        c->step += ran;
        if (h > 0) {
            if (int rc = apply_step_splits(c)) return rc;
            c->spec_len = 1;
            if (int rc = run_steps(c, n - ran)) return rc;   // the topology changed: no replay
        } else if (c->hcount[CNT_ERR] & DERR_SCAN_WAIT) {
            return cem_fail(c, CEM_ETIMEOUT, "a scan's bounded look-back wait gave up");
        }
    }
    if (int rc = cem_launch_check_finite(c)) return rc;
    if (int rc = sync_counts(c)) return rc;
    if (int rc = check_tma_wait(c)) return rc;
    if (c->hcount[CNT_SCRATCH1]) return cem_fail(c, CEM_ENONFINITE, "non-finite displacement");
    return CEM_OK;
}

int cem_profile(cem_ctx* c, int enable) {
    if (!c) return CEM_EINVAL;
    if (int rc = select_device(c)) return rc;
    if (int rc = prof_resolve(c)) return rc;
    if (enable) {
        for (int q = 0; q < CEM_KERNEL_COUNT; ++q) {
            c->prof_ms[q] = 0.0;
            c->prof_n[q] = 0;
        }
        c->n_launch = 0;
    }
    c->prof = enable > 0;
    c->prof_every = enable > 0 ? enable : 1;
    c->prof_now = false;
    return CEM_OK;
}

int cem_profile_read(cem_ctx* c, double* ms, int64_t* launches, int n, int64_t* total_launches) {
    if (!c || n < 0) return CEM_EINVAL;
    if (int rc = select_device(c)) return rc;
    if (int rc = prof_resolve(c)) return rc;
    for (int q = 0; q < n && q < CEM_KERNEL_COUNT; ++q) {
        if (ms) ms[q] = c->prof_ms[q];
        if (launches) launches[q] = c->prof_n[q];
    }
    if (total_launches) *total_launches = c->n_launch;
    return CEM_OK;
}

int cem_energy(cem_ctx* c, cem_energy_t* out) {
    if (!c || !out) return CEM_EINVAL;
    if (!c->material) return cem_fail(c, CEM_ESTATE, "no material");
    if (int rc = select_device(c)) return rc;
    int rc;
    if ((rc = cem_launch_split_u(c)) || (rc = cem_launch_strain(c)) || (rc = cem_launch_edge_stress(c))) return rc;
    double r[4];
    if ((rc = cem_energy_reduce(c, r)) || (rc = cem_launch_pred_u(c))) return rc;
    double Ud = 0.0;
    CEM_CK(c, cudaMemcpy(&Ud, c->Ud, sizeof(double), cudaMemcpyDeviceToHost));
    out->kinetic = r[0];
    out->ext_work = r[1];
    out->strain = r[3];
    out->dissipated = Ud;
    out->modified = r[0] + r[3] - r[1] - c->dt * c->dt / 8.0 * r[2];
    out->step = c->step;
    out->time = (double)c->step * c->dt;
    out->n_split = c->n_split_run;
    return CEM_OK;
}

int cem_energy_instance(cem_ctx* c, int64_t instance, cem_energy_t* out) {
    if (!c || !out) return CEM_EINVAL;
    if (instance < 0 || instance >= c->n_inst) return cem_fail(c, CEM_EINVAL, "instance out of range");
    if (!c->material) return cem_fail(c, CEM_ESTATE, "no material");
    if (int rc = select_device(c)) return rc;
    int rc;
    if ((rc = cem_launch_split_u(c)) || (rc = cem_launch_strain(c)) || (rc = cem_launch_edge_stress(c))) return rc;
    double r[5];
    if ((rc = cem_energy_reduce_instance(c, (int)instance, r)) || (rc = cem_launch_pred_u(c))) return rc;
    const double dt = c->inst_dt[instance];
    int64_t nsplit = 0;
    if (c->n_inst > 1) {
        // run-time splits of this specimen: counted on the host from the crack state
        std::vector<uint8_t> sd(c->T0);
        std::vector<int> st(c->T0);
        CEM_CK(c, cudaMemcpy(sd.data(), c->side, c->T0, cudaMemcpyDeviceToHost));
        CEM_CK(c, cudaMemcpy(st.data(), c->split_step, c->T0 * sizeof(int), cudaMemcpyDeviceToHost));
        for (int64_t t = 0; t < c->T0; ++t)
            if (sd[t] && st[t] >= 0 && c->h_tet_inst[t] == instance) ++nsplit;
    } else {
        nsplit = c->n_split_run;
    }
    out->kinetic = r[0];
    out->ext_work = r[1];
    out->strain = r[3];
    out->dissipated = r[4];
    out->modified = r[0] + r[3] - r[1] - dt * dt / 8.0 * r[2];
    out->step = c->step;
    out->time = (double)c->step * dt;
    out->n_split = nsplit;
    return CEM_OK;
}

int cem_crack_state(cem_ctx* c, int64_t* n_split, int32_t* tet, int8_t* pattern, uint8_t* side, int64_t* step,
                    double* G, int64_t cap) {
    if (!c || !n_split) return CEM_EINVAL;
    if (c->elem_type != CEM_ELEM_TET4) {   // hexahedral meshes never split
        *n_split = 0;
        return CEM_OK;
    }
    if (int rc = select_device(c)) return rc;
    const int64_t T0 = c->T0;
    std::vector<uint8_t> sd(T0);
    std::vector<int> st(T0);
    std::vector<double> g(T0);
    CEM_CK(c, cudaMemcpyAsync(sd.data(), c->side, T0, cudaMemcpyDeviceToHost, c->stream));
    CEM_CK(c, cudaMemcpyAsync(st.data(), c->split_step, T0 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CEM_CK(c, cudaMemcpyAsync(g.data(), c->split_G, T0 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    std::vector<std::pair<int, int>> rec;
    for (int64_t t = 0; t < T0; ++t)
        if (sd[t]) rec.push_back({st[t], (int)t});
    std::sort(rec.begin(), rec.end());
    *n_split = (int64_t)rec.size();
    const int64_t m = std::min<int64_t>(cap, (int64_t)rec.size());
    for (int64_t q = 0; q < m; ++q) {
        const int t = rec[q].second;
        if (tet) tet[q] = t;
        if (pattern) pattern[q] = (int8_t)(__builtin_popcount(sd[t]) == 2 ? CEM_PATTERN_I : CEM_PATTERN_II);
        if (side) side[q] = sd[t];
        if (step) step[q] = rec[q].first;
        if (G) G[q] = g[t];
    }
    return CEM_OK;
}

int cem_get_field(cem_ctx* c, int which, double* out, int64_t cap, int64_t* n_nodes) {
    if (!c) return CEM_EINVAL;
    if (n_nodes) *n_nodes = c->N;
    if (!out) return CEM_OK;
    if (cap < 3 * c->N) return cem_fail(c, CEM_EINVAL, "output buffer too small");
    const double* src = which == CEM_FIELD_U ? c->u : which == CEM_FIELD_V ? c->v : which == CEM_FIELD_A ? c->a
                      : which == CEM_FIELD_X ? c->X : nullptr;
    if (!src) return cem_fail(c, CEM_EINVAL, "unknown field");
    if (int rc = select_device(c)) return rc;
    std::vector<double> tmp(3 * c->N);
    for (int k = 0; k < 3; ++k)
        CEM_CK(c, cudaMemcpyAsync(tmp.data() + k * c->N, src + k * c->Nc, c->N * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream));
    std::vector<int> at;   // storage index of every creation id (renumbered nodes)
    if (c->renumbered) {
        at.resize(c->N);
        CEM_CK(c, cudaMemcpyAsync(at.data(), c->int_of_ext, c->N * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    }
    CEM_CK(c, cudaStreamSynchronize(c->stream));
    for (int64_t i = 0; i < c->N; ++i) {
        const int64_t j = c->renumbered ? at[i] : i;
        for (int k = 0; k < 3; ++k) out[3 * i + k] = tmp[k * c->N + j];
    }
    return CEM_OK;
}

int cem_info(cem_ctx* c, cem_info_t* out) {
    if (!c || !out) return CEM_EINVAL;
    out->n_nodes = c->N;
    out->n_tets = c->T;
    out->n_active_tets = c->n_active;
    out->n_edges = c->E;
    out->n_candidates = c->n_cand;
    out->n_orig_edges = c->E0;
    out->dt = c->dt;
    out->h_min = c->h_min;
    out->device_bytes = c->bytes;
    out->n_reorder = c->n_reorder;
    out->persistent_blocks = c->persist_blocks;
    return CEM_OK;
}

int cem_destroy(cem_ctx* c) {
    if (!c) return CEM_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->side_stream) {
        cudaStreamSynchronize(c->side_stream);
        cudaStreamDestroy(c->side_stream);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->cap_stream) {
        cudaStreamSynchronize(c->cap_stream);
        cudaStreamDestroy(c->cap_stream);
    }
    for (void* p : c->allocs) {
        if (c->free_fn) c->free_fn(p, (void*)c->stream, c->alloc_user);
        else cudaFree(p);
    }
    for (auto& r : c->ev_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->hcount) cudaFreeHost(c->hcount);
    if (c->hred) cudaFreeHost(c->hred);
    delete c;
    return CEM_OK;
}

const char* cem_last_error(const cem_ctx* c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

}  // extern "C"
