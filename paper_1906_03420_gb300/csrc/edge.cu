// Edge isomorphism by the line-graph transform (Sec. VII-A).
//
// The paper reduces edge isomorphism to vertex isomorphism: every edge of G
// becomes a vertex of G', and every pair of edges that meet at a vertex of G
// becomes an edge of G'.  Q is transformed the same way, Q' is matched in G'
// by the ordinary path, and the matches of Q' are read back as edge maps.
// Labels, which the paper leaves open, are carried over so that nothing of
// the original labelling is lost:
//   - vertex i of G' (edge i of G, {a, b}, label l) gets a dense id of the
//     triple (l, min(r(a), r(b)), max(r(a), r(b))), where r is the rank of a
//     vertex label among G's sorted distinct vertex labels;
//   - the edge of G' between edges i and j of G that meet at vertex v gets
//     r(v).
// A simple graph's edges meet at one vertex at most, so G' is simple.  The id
// of a G' vertex is the position of its edge in the caller's list, and the
// id of a Q' vertex is that of its query edge.  The reverse transform is
// therefore the identity: a match row lists data edge ids, column j for query
// edge j.
//
// Everything here runs on the host.  Device work is the library's ordinary
// graph build and query on G' and Q'.
#include <algorithm>
#include <array>
#include <climits>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "runtime.h"

using namespace gsi;

struct gsi_edge_graph {
    int32_t n = 0;
    int64_t m = 0;
    std::vector<int32_t> vlab, src, dst, elab;         // G, as given
    std::vector<int32_t> vlabels;                       // sorted distinct vertex labels of G
    std::vector<std::array<int32_t, 3>> keys;           // sorted distinct line-vertex label triples
    int64_t lm = 0;                                     // |E(G')|
    gsi_graph *line = nullptr;                          // G' on the device (NULL: host only)
};

namespace {

int32_t rank_of(const std::vector<int32_t> &sorted, int32_t label) {
    auto it = std::lower_bound(sorted.begin(), sorted.end(), label);
    return (it != sorted.end() && *it == label) ? (int32_t)(it - sorted.begin()) : -1;
}

std::array<int32_t, 3> triple(int32_t l, int32_t ra, int32_t rb) {
    return {l, std::min(ra, rb), std::max(ra, rb)};
}

// Incident edge ids of each vertex (CSR over 0..n-1, ids ascending).
void incidence(int32_t n, const int32_t *src, const int32_t *dst, int64_t m, std::vector<int64_t> &start,
               std::vector<int32_t> &inc) {
    start.assign((size_t)n + 1, 0);
    for (int64_t e = 0; e < m; ++e) { start[(size_t)src[e] + 1]++; start[(size_t)dst[e] + 1]++; }
    for (int32_t v = 0; v < n; ++v) start[(size_t)v + 1] += start[(size_t)v];
    inc.resize((size_t)(2 * m));
    std::vector<int64_t> cur(start.begin(), start.end() - 1);
    for (int64_t e = 0; e < m; ++e) {
        inc[(size_t)cur[(size_t)src[e]]++] = (int32_t)e;
        inc[(size_t)cur[(size_t)dst[e]]++] = (int32_t)e;
    }
}

// Check G and fill the label tables and |E(G')|.
gsi_status prepare(gsi_edge_graph *eg) {
    const int32_t n = eg->n;
    const int64_t m = eg->m;
    for (int64_t e = 0; e < m; ++e) {
        const int32_t a = eg->src[(size_t)e], b = eg->dst[(size_t)e];
        if (a < 0 || a >= n || b < 0 || b >= n) {
            set_error("gsi_edge_graph_create: vertex id out of range");
            return GSI_EINVAL;
        }
        if (a == b) {
            set_error("gsi_edge_graph_create: self-loop");
            return GSI_EINVAL;
        }
        if (eg->elab[(size_t)e] < 0) {
            set_error("gsi_edge_graph_create: negative edge label");
            return GSI_EINVAL;
        }
    }
    {
        std::vector<uint64_t> pairs((size_t)m);
        for (int64_t e = 0; e < m; ++e) {
            const uint32_t a = (uint32_t)eg->src[(size_t)e], b = (uint32_t)eg->dst[(size_t)e];
            pairs[(size_t)e] = ((uint64_t)std::min(a, b) << 32) | std::max(a, b);
        }
        std::sort(pairs.begin(), pairs.end());
        if (std::adjacent_find(pairs.begin(), pairs.end()) != pairs.end()) {
            set_error("gsi_edge_graph_create: the same vertex pair given twice");
            return GSI_EINVAL;
        }
    }
    eg->vlabels = eg->vlab;
    std::sort(eg->vlabels.begin(), eg->vlabels.end());
    eg->vlabels.erase(std::unique(eg->vlabels.begin(), eg->vlabels.end()), eg->vlabels.end());
    std::vector<int32_t> r((size_t)n);
    for (int32_t v = 0; v < n; ++v) r[(size_t)v] = rank_of(eg->vlabels, eg->vlab[(size_t)v]);
    eg->keys.resize((size_t)m);
    for (int64_t e = 0; e < m; ++e)
        eg->keys[(size_t)e] = triple(eg->elab[(size_t)e], r[(size_t)eg->src[(size_t)e]], r[(size_t)eg->dst[(size_t)e]]);
    std::sort(eg->keys.begin(), eg->keys.end());
    eg->keys.erase(std::unique(eg->keys.begin(), eg->keys.end()), eg->keys.end());
    if (eg->keys.size() > 65535) {
        set_error("gsi_edge_graph_create: more than 65535 distinct (edge label, endpoint labels) triples");
        return GSI_EINVAL;
    }
    std::vector<int64_t> deg((size_t)n, 0);
    for (int64_t e = 0; e < m; ++e) { deg[(size_t)eg->src[(size_t)e]]++; deg[(size_t)eg->dst[(size_t)e]]++; }
    uint64_t lm = 0;
    for (int32_t v = 0; v < n; ++v) lm += (uint64_t)deg[(size_t)v] * (uint64_t)(deg[(size_t)v] - 1) / 2;
    if (lm >= ((uint64_t)1 << 31)) {
        set_error("gsi_edge_graph_create: the line graph has 2^31 edges or more (sum over vertices of "
                  "deg(deg-1)/2); the graph build holds at most 2^31 - 1");
        return GSI_EINVAL;
    }
    eg->lm = (int64_t)lm;
    return GSI_OK;
}

int32_t key_id(const gsi_edge_graph *eg, const std::array<int32_t, 3> &t) {
    auto it = std::lower_bound(eg->keys.begin(), eg->keys.end(), t);
    return (it != eg->keys.end() && *it == t) ? (int32_t)(it - eg->keys.begin()) : -1;
}

// G' into the given arrays (any may be null); edges beyond cap are not written.
void line_of_graph(const gsi_edge_graph *eg, int32_t *lvlab, int32_t *lsrc, int32_t *ldst, int32_t *lelab,
                   int64_t cap) {
    const int32_t n = eg->n;
    const int64_t m = eg->m;
    if (lvlab) {
        for (int64_t e = 0; e < m; ++e) {
            const int32_t ra = rank_of(eg->vlabels, eg->vlab[(size_t)eg->src[(size_t)e]]);
            const int32_t rb = rank_of(eg->vlabels, eg->vlab[(size_t)eg->dst[(size_t)e]]);
            lvlab[e] = key_id(eg, triple(eg->elab[(size_t)e], ra, rb));
        }
    }
    if (!(lsrc || ldst || lelab) || cap <= 0) return;
    std::vector<int64_t> start;
    std::vector<int32_t> inc;
    incidence(n, eg->src.data(), eg->dst.data(), m, start, inc);
    int64_t p = 0;
    for (int32_t v = 0; v < n && p < cap; ++v) {
        const int32_t rv = rank_of(eg->vlabels, eg->vlab[(size_t)v]);
        for (int64_t i = start[(size_t)v]; i < start[(size_t)v + 1] && p < cap; ++i)
            for (int64_t j = i + 1; j < start[(size_t)v + 1] && p < cap; ++j, ++p) {
                if (lsrc) lsrc[p] = inc[(size_t)i];
                if (ldst) ldst[p] = inc[(size_t)j];
                if (lelab) lelab[p] = rv;
            }
    }
}

// Q' of a validated query: qm vertices, edges between query edges that share
// a query vertex.  Labels absent from G become values no line vertex or edge
// carries (-1 for a vertex, INT32_MAX for an edge).
void line_of_query(const gsi_edge_graph *eg, const QueryGraph &q, std::vector<int32_t> &lvlab,
                   std::vector<int32_t> &lsrc, std::vector<int32_t> &ldst, std::vector<int32_t> &lelab) {
    lvlab.assign((size_t)q.qm, -1);
    for (int32_t e = 0; e < q.qm; ++e) {
        const int32_t ra = rank_of(eg->vlabels, q.vl[(size_t)q.src[(size_t)e]]);
        const int32_t rb = rank_of(eg->vlabels, q.vl[(size_t)q.dst[(size_t)e]]);
        if (ra >= 0 && rb >= 0) lvlab[(size_t)e] = key_id(eg, triple(q.lab[(size_t)e], ra, rb));
    }
    std::vector<int64_t> start;
    std::vector<int32_t> inc;
    incidence(q.k, q.src.data(), q.dst.data(), q.qm, start, inc);
    lsrc.clear(); ldst.clear(); lelab.clear();
    for (int32_t u = 0; u < q.k; ++u) {
        const int32_t ru = rank_of(eg->vlabels, q.vl[(size_t)u]);
        for (int64_t i = start[(size_t)u]; i < start[(size_t)u + 1]; ++i)
            for (int64_t j = i + 1; j < start[(size_t)u + 1]; ++j) {
                lsrc.push_back(inc[(size_t)i]);
                ldst.push_back(inc[(size_t)j]);
                lelab.push_back(ru >= 0 ? ru : INT32_MAX);
            }
    }
}

gsi_status edge_query(const gsi_edge_graph *eg, const int32_t *qvlab, int32_t k, const int32_t *qsrc,
                      const int32_t *qdst, const int32_t *qelab, int32_t qm, std::vector<int32_t> &lvlab,
                      std::vector<int32_t> &lsrc, std::vector<int32_t> &ldst, std::vector<int32_t> &lelab) {
    if (qm < 1 || qm > GSI_MAX_QUERY_VERTICES) {
        set_error("edge query: need 1 <= edges <= 32 (one line-graph vertex per query edge)");
        return GSI_EINVAL;
    }
    QueryGraph q;
    GSI_TRY(validate_query(qvlab, k, qsrc, qdst, qelab, qm, &q));
    line_of_query(eg, q, lvlab, lsrc, ldst, lelab);
    return GSI_OK;
}

}  // namespace

extern "C" {

gsi_status gsi_edge_graph_create(const int32_t *vlab, int32_t n, const int32_t *src, const int32_t *dst,
                                 const int32_t *elab, int64_t m, const gsi_graph_opts *opts, int32_t flags,
                                 gsi_edge_graph **out) {
    GSI_API_BEGIN
    if (!out) {
        set_error("gsi_edge_graph_create: null out");
        return GSI_EINVAL;
    }
    *out = nullptr;
    if (n < 1 || m < 1 || m >= ((int64_t)1 << 31)) {
        set_error("gsi_edge_graph_create: need n >= 1 and 1 <= m < 2^31");
        return GSI_EINVAL;
    }
    if (!vlab || !src || !dst || !elab) {
        set_error("gsi_edge_graph_create: null array");
        return GSI_EINVAL;
    }
    if (flags & ~GSI_EDGE_HOST_ONLY) {
        set_error("gsi_edge_graph_create: unknown flag");
        return GSI_EINVAL;
    }
    std::unique_ptr<gsi_edge_graph> eg(new gsi_edge_graph());
    eg->n = n;
    eg->m = m;
    eg->vlab.assign(vlab, vlab + n);
    eg->src.assign(src, src + m);
    eg->dst.assign(dst, dst + m);
    eg->elab.assign(elab, elab + m);
    GSI_TRY(prepare(eg.get()));
    if (!(flags & GSI_EDGE_HOST_ONLY)) {
        std::vector<int32_t> lvlab((size_t)m), lsrc((size_t)eg->lm + 1), ldst((size_t)eg->lm + 1),
            lelab((size_t)eg->lm + 1);
        line_of_graph(eg.get(), lvlab.data(), lsrc.data(), ldst.data(), lelab.data(), eg->lm);
        GSI_TRY(gsi_graph_create(lvlab.data(), (int32_t)m, lsrc.data(), ldst.data(), lelab.data(), eg->lm, opts,
                                 &eg->line));
    }
    *out = eg.release();
    return GSI_OK;
    GSI_API_END
}

void gsi_edge_graph_destroy(gsi_edge_graph *g) {
    if (!g) return;
    gsi_graph_destroy(g->line);
    delete g;
}

gsi_status gsi_edge_graph_line(const gsi_edge_graph *g, int32_t *lvlab, int32_t *lsrc, int32_t *ldst,
                               int32_t *lelab, int64_t cap, int32_t *ln, int64_t *lm) {
    GSI_API_BEGIN
    if (!g) {
        set_error("gsi_edge_graph_line: null graph");
        return GSI_EINVAL;
    }
    if (ln) *ln = (int32_t)g->m;
    if (lm) *lm = g->lm;
    line_of_graph(g, lvlab, lsrc, ldst, lelab, std::min<int64_t>(cap, g->lm));
    return GSI_OK;
    GSI_API_END
}

gsi_status gsi_edge_graph_device(const gsi_edge_graph *g, gsi_graph **line) {
    if (!g || !line) {
        set_error("gsi_edge_graph_device: null argument");
        return GSI_EINVAL;
    }
    *line = g->line;
    return GSI_OK;
}

gsi_status gsi_edge_query_line(const gsi_edge_graph *g, const int32_t *qvlab, int32_t k, const int32_t *qsrc,
                               const int32_t *qdst, const int32_t *qelab, int32_t qm, int32_t *lvlab,
                               int32_t *lsrc, int32_t *ldst, int32_t *lelab, int32_t cap, int32_t *lk,
                               int32_t *lqm) {
    GSI_API_BEGIN
    if (!g) {
        set_error("gsi_edge_query_line: null graph");
        return GSI_EINVAL;
    }
    std::vector<int32_t> vl, s, d, l;
    GSI_TRY(edge_query(g, qvlab, k, qsrc, qdst, qelab, qm, vl, s, d, l));
    if (lk) *lk = (int32_t)vl.size();
    if (lqm) *lqm = (int32_t)s.size();
    if (lvlab) std::memcpy(lvlab, vl.data(), sizeof(int32_t) * vl.size());
    const size_t c = std::min<size_t>(s.size(), (size_t)std::max(cap, 0));
    if (lsrc) std::memcpy(lsrc, s.data(), sizeof(int32_t) * c);
    if (ldst) std::memcpy(ldst, d.data(), sizeof(int32_t) * c);
    if (lelab) std::memcpy(lelab, l.data(), sizeof(int32_t) * c);
    return GSI_OK;
    GSI_API_END
}

gsi_status gsi_edge_query_run(gsi_edge_graph *g, const int32_t *qvlab, int32_t k, const int32_t *qsrc,
                              const int32_t *qdst, const int32_t *qelab, int32_t qm, const gsi_query_opts *opts,
                              gsi_result **out) {
    GSI_API_BEGIN
    if (!g || !out) {
        set_error("gsi_edge_query_run: null graph or out");
        return GSI_EINVAL;
    }
    *out = nullptr;
    if (!g->line) {
        set_error("gsi_edge_query_run: the edge graph was created host-only");
        return GSI_EINVAL;
    }
    if (opts && opts->semantics != GSI_ISOMORPHISM) {
        set_error("gsi_edge_query_run: edge queries take GSI_ISOMORPHISM semantics only");
        return GSI_EINVAL;
    }
    std::vector<int32_t> vl, s, d, l;
    GSI_TRY(edge_query(g, qvlab, k, qsrc, qdst, qelab, qm, vl, s, d, l));
    return gsi_query_run(g->line, vl.data(), (int32_t)vl.size(), s.data(), d.data(), l.data(), (int32_t)s.size(),
                         opts, out);
    GSI_API_END
}

}  // extern "C"
