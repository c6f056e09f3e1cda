// Factorisation-formula front end: the operator vocabulary of Table I
// (DFT(n), I(n), A ⊗ B, A · B, twiddle(N, M), Permute(N, K)), parsed on the
// host and checked to denote DFT_N by the Cooley-Tukey identity of Eq. 2,
//     DFT_N = (DFT_K ⊗ I_M) · twiddle(N, M) · (I_K ⊗ DFT_M) · Permute(N, K),  N = K M,
// applied recursively (either DFT factor may itself be such a product; Eq. 1
// is the case N = 4), or its transpose Permute(N, M) · (I_K ⊗ DFT_M) ·
// twiddle(N, M) · (DFT_K ⊗ I_M) (decimation in frequency), or Pease's
// constant-geometry product for N = R^t (as_pease below).  twiddle(N, M) is the diagonal D^N_M and Permute(N, K)
// the stride permutation Pi^N_K of Eq. 2 (their argument order follows the
// subscripts of Eq. 2).  A checked formula then selects the execution plan:
// its DFT leaves, in the order the product applies them (rightmost first),
// are the radix schedule of a single-pass plan, and its outermost split K x M
// is the k_outer of a two-pass plan.
//
// Syntax (after the paper's grammar, Sec. IV-A): factors joined by ⊗ (or the
// ASCII word `kron`) and · (or `*` or `.`), both right-associative at one
// precedence level, parentheses, integer arguments.  A formula may be written
// as a program line, `var result = <formula> · InputComplex;`: a trailing
// identifier (the input vector) and the `var name =` prefix and `;` are
// accepted and ignored.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"

namespace gbfft {
namespace {

enum NodeKind { kDft, kIdent, kTwiddle, kPermute, kKron, kProd, kInput };

struct Node {
    NodeKind kind;
    int64_t a = 0, b = 0;           // integer arguments
    std::unique_ptr<Node> l, r;     // operands of kKron / kProd
};

struct Parser {
    const char* s;
    size_t pos = 0;
    std::string err;

    explicit Parser(const char* text) : s(text) {}

    void skip() {
        while (s[pos] == ' ' || s[pos] == '\t' || s[pos] == '\n' || s[pos] == '\r') ++pos;
    }
    bool fail(const std::string& m) {
        if (err.empty()) err = m + " at offset " + std::to_string(pos);
        return false;
    }
    bool accept(const char* tok) {
        skip();
        const size_t n = std::strlen(tok);
        if (std::strncmp(s + pos, tok, n) == 0) {
            pos += n;
            return true;
        }
        return false;
    }
    static bool ident_char(char c) {
        return (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || (c >= '0' && c <= '9') || c == '_';
    }
    bool word(std::string* out) {
        skip();
        const size_t b = pos;
        if (!((s[pos] >= 'a' && s[pos] <= 'z') || (s[pos] >= 'A' && s[pos] <= 'Z') || s[pos] == '_')) return false;
        while (ident_char(s[pos])) ++pos;
        *out = std::string(s + b, pos - b);
        return true;
    }
    bool integer(int64_t* v) {
        skip();
        if (s[pos] < '0' || s[pos] > '9') return fail("expected an integer");
        int64_t x = 0;
        while (s[pos] >= '0' && s[pos] <= '9') {
            x = x * 10 + (s[pos] - '0');
            if (x > ((int64_t)1 << 40)) return fail("integer too large");
            ++pos;
        }
        *v = x;
        return true;
    }
    // Binary operator: 1 = Kronecker, 2 = product, 0 = none.
    int op() {
        skip();
        const size_t save = pos;
        if (accept("\xE2\x8A\x97")) return 1;  // ⊗
        if (accept("\xC2\xB7")) return 2;      // ·
        if (accept("*") || accept(".")) return 2;
        std::string w;
        if (word(&w) && w == "kron") return 1;
        pos = save;
        return 0;
    }
    bool args(int count, int64_t* a, int64_t* b) {
        if (!accept("(")) return fail("expected '('");
        if (!integer(a)) return false;
        if (count == 2) {
            if (!accept(",")) return fail("expected ','");
            if (!integer(b)) return false;
        }
        if (!accept(")")) return fail("expected ')'");
        return true;
    }
    std::unique_ptr<Node> primary() {
        skip();
        if (accept("(")) {
            auto e = expr();
            if (!e) return nullptr;
            if (!accept(")")) {
                fail("expected ')'");
                return nullptr;
            }
            return e;
        }
        std::string w;
        if (!word(&w)) {
            fail("expected a factor");
            return nullptr;
        }
        auto n = std::make_unique<Node>();
        bool ok = true;
        if (w == "DFT" || w == "dft") {
            n->kind = kDft;
            ok = args(1, &n->a, nullptr);
        } else if (w == "I" || w == "identity") {
            n->kind = kIdent;
            ok = args(1, &n->a, nullptr);
        } else if (w == "twiddle") {
            n->kind = kTwiddle;
            ok = args(2, &n->a, &n->b);
        } else if (w == "Permute" || w == "permute") {
            n->kind = kPermute;
            ok = args(2, &n->a, &n->b);
        } else {
            n->kind = kInput;  // an input vector such as InputComplex
        }
        return ok ? std::move(n) : nullptr;
    }
    // expr := primary ((⊗ | ·) expr)?   (right-associative, one precedence level)
    std::unique_ptr<Node> expr() {
        auto l = primary();
        if (!l) return nullptr;
        const int o = op();
        if (o == 0) return l;
        auto r = expr();
        if (!r) return nullptr;
        auto n = std::make_unique<Node>();
        n->kind = o == 1 ? kKron : kProd;
        n->l = std::move(l);
        n->r = std::move(r);
        return n;
    }
    std::unique_ptr<Node> program() {
        skip();
        const size_t save = pos;
        std::string w;
        if (word(&w) && w == "var") {  // var <name> = <formula> ;
            std::string name;
            if (!word(&name) || !accept("=")) {
                fail("expected 'var <name> ='");
                return nullptr;
            }
        } else {
            pos = save;
        }
        auto e = expr();
        if (!e) return nullptr;
        accept(";");
        skip();
        if (s[pos] != '\0') {
            fail("unexpected text after the formula");
            return nullptr;
        }
        return e;
    }
};

// Matrix dimension of a node (0 if ill-formed, with a message).
int64_t dim(const Node* n, std::string* err) {
    switch (n->kind) {
        case kDft:
        case kIdent:
            if (n->a < 1) return *err = "DFT(n) and I(n) need n >= 1", 0;
            return n->a;
        case kTwiddle:
        case kPermute:
            if (n->a < 1 || n->b < 1 || n->a % n->b != 0)
                return *err = "twiddle(N, M) and Permute(N, K) need a divisor of N", 0;
            return n->a;
        case kInput:
            return *err = "an input vector may only be the last factor of the formula", 0;
        case kKron: {
            const int64_t a = dim(n->l.get(), err), b = dim(n->r.get(), err);
            if (!a || !b) return 0;
            if (a > ((int64_t)1 << 40) / b) return *err = "dimension too large", 0;
            return a * b;
        }
        case kProd: {
            const int64_t a = dim(n->l.get(), err), b = dim(n->r.get(), err);
            if (!a || !b) return 0;
            if (a != b) return *err = "factors of a product must have equal dimensions", 0;
            return a;
        }
    }
    return 0;
}

void flatten_product(const Node* n, std::vector<const Node*>* out) {
    if (n->kind == kProd) {
        flatten_product(n->l.get(), out);
        flatten_product(n->r.get(), out);
    } else {
        out->push_back(n);
    }
}

struct DftForm {
    int64_t n = 0;
    int64_t k_top = 0;            // outermost split N = K * M (0: a single DFT(n) leaf)
    bool bare = false;            // the outermost split is Eq. 2's own order over DFT(K), DFT(M) leaves
    bool transposed = false;      // the outermost split is the transposed (decimation-in-frequency) form
    bool pease = false;           // the whole formula is Pease's constant-geometry product
    std::vector<int64_t> leaves;  // DFT leaf sizes in application order
};

bool as_dft(const Node* n, DftForm* f, std::string* err);

// The transpose of Eq. 2 (DFT_N is symmetric, D diagonal, (Pi^N_K)^T = Pi^N_M):
//     DFT_N = Permute(N, M) · (I_K ⊗ DFT_M) · twiddle(N, M) · (DFT_K ⊗ I_M),
// the decimation-in-frequency order; DFT_K runs first, then DFT_M.
bool as_dft_transposed(const std::vector<const Node*>& fs, DftForm* f, std::string* err) {
    const Node *f1 = fs[0], *f2 = fs[1], *f3 = fs[2], *f4 = fs[3];
    if (f2->kind != kKron || f2->l->kind != kIdent)
        return *err = "transposed form: second factor must be (I_K (x) DFT_M)", false;
    if (f3->kind != kTwiddle) return *err = "transposed form: third factor must be twiddle(N, M)", false;
    if (f4->kind != kKron || f4->r->kind != kIdent)
        return *err = "transposed form: fourth factor must be (DFT_K (x) I_M)", false;
    DftForm x, y;
    if (!as_dft(f4->l.get(), &x, err) || !as_dft(f2->r.get(), &y, err)) return false;
    const int64_t K = x.n, M = y.n, N = K * M;
    if (f4->r->a != M || f2->l->a != K)
        return *err = "transposed form: identity sizes must match the DFT factors", false;
    if (f3->a != N || f3->b != M) return *err = "transposed form: third factor must be twiddle(N, M)", false;
    if (f1->a != N || f1->b != M) return *err = "transposed form: first factor must be Permute(N, M)", false;
    f->n = N;
    f->k_top = K;
    f->bare = false;  // the split is Eq. 2's, but the factors run in the other order
    f->transposed = true;
    f->leaves = x.leaves;  // DFT_K first, then DFT_M
    f->leaves.insert(f->leaves.end(), y.leaves.begin(), y.leaves.end());
    return true;
}

bool is_kind(const Node* n, NodeKind k, int64_t a, int64_t b = -1) {
    return n->kind == k && n->a == a && (b < 0 || n->b == b);
}

// I(size), written as one identity or as the Kronecker product of identities.
bool is_identity(const Node* n, int64_t size) {
    if (n->kind == kIdent) return n->a == size;
    if (n->kind != kKron) return false;
    std::string e;
    const int64_t a = dim(n->l.get(), &e);
    return a > 0 && size % a == 0 && is_identity(n->l.get(), a) && is_identity(n->r.get(), size / a);
}

// Whether the product of `fs` is the base-R digit reversal of length N,
//     Rev_N = (I(R) ⊗ Rev_{N/R}) · Permute(N, R),  Rev_R = I(R)
// (with Rev_{R^2} = Permute(R^2, R) accepted without its identity factor).
bool is_reversal(const std::vector<const Node*>& fs, int64_t N, int64_t R) {
    if (N == R) return fs.empty() || (fs.size() == 1 && is_identity(fs[0], R));
    if (fs.size() == 1) return N == R * R && is_kind(fs[0], kPermute, N, R);
    if (fs.size() != 2 || !is_kind(fs[1], kPermute, N, R)) return false;
    const Node* k = fs[0];
    if (k->kind != kKron || !is_identity(k->l.get(), R)) return false;
    std::vector<const Node*> inner;
    flatten_product(k->r.get(), &inner);
    return is_reversal(inner, N / R, R);
}

// Pease's constant-geometry form of DFT_N, N = R^t, t >= 2 (Eq. 2 with K = R
// unrolled over the digits, the permutations gathered into one digit reversal
// applied first):
//     DFT_N = G_t · ... · G_1 · Rev_N,
//     G_s   = (DFT(R) ⊗ I(N/R)) · (twiddle(R^s, R^(s-1)) ⊗ I(R^(t-s))) · Permute(N, R),
// where G_t's twiddle factor may be written twiddle(N, N/R) alone (its
// identity is I(1)).  Its DFT leaves are t copies of DFT(R).
bool as_pease(const std::vector<const Node*>& fs, DftForm* f, std::string* err) {
    const Node* f0 = fs[0];
    if (f0->kind != kKron || f0->l->kind != kDft || f0->r->kind != kIdent || f0->l->a < 2)
        return *err = "Pease form: first factor must be (DFT(R) (x) I(N/R))", false;
    const int64_t R = f0->l->a, N = R * f0->r->a;
    int t = 0;
    for (int64_t m = 1; m < N; m *= R) ++t;
    int64_t p = 1;
    for (int i = 0; i < t; ++i) p *= R;
    if (p != N || t < 2) return *err = "Pease form: N must be a power of R with at least two stages", false;
    if (fs.size() < (size_t)(3 * t)) return *err = "Pease form: three factors per stage, t stages for N = R^t", false;
    int64_t rs = N;  // R^s for the stage s = t - i
    for (int i = 0; i < t; ++i, rs /= R) {
        const int s = t - i;
        const Node *a = fs[3 * i], *b = fs[3 * i + 1], *c = fs[3 * i + 2];
        if (a->kind != kKron || !is_kind(a->l.get(), kDft, R) || !is_identity(a->r.get(), N / R))
            return *err = "Pease form, stage " + std::to_string(s) + ": expected (DFT(R) (x) I(N/R))", false;
        const bool tw_ok =
            (b->kind == kKron && is_kind(b->l.get(), kTwiddle, rs, rs / R) && is_identity(b->r.get(), N / rs)) ||
            (rs == N && is_kind(b, kTwiddle, N, N / R));
        if (!tw_ok)
            return *err = "Pease form, stage " + std::to_string(s) + ": expected (twiddle(R^s, R^(s-1)) (x) I(R^(t-s)))",
                   false;
        if (!is_kind(c, kPermute, N, R))
            return *err = "Pease form, stage " + std::to_string(s) + ": expected Permute(N, R)", false;
    }
    const std::vector<const Node*> rest(fs.begin() + 3 * t, fs.end());
    if (!is_reversal(rest, N, R))
        return *err = "Pease form: the stages must be followed by the digit reversal "
                      "Rev_N = (I(R) (x) Rev_(N/R)) . Permute(N, R), Rev_R = I(R)",
               false;
    f->n = N;
    f->k_top = 0;
    f->bare = false;
    f->transposed = false;
    f->pease = true;
    f->leaves.assign((size_t)t, R);
    return true;
}

// Whether n denotes DFT_N: a DFT(n) leaf, Eq. 2's four factors (or their
// transpose) with DFT factors that themselves denote DFTs, or Pease's form.
bool as_dft(const Node* n, DftForm* f, std::string* err) {
    if (n->kind == kDft) {
        f->n = n->a;
        f->k_top = 0;
        f->leaves = {n->a};
        return true;
    }
    if (n->kind != kProd) return *err = "not a DFT: expected DFT(n) or a product of Eq. 2's four factors", false;
    std::vector<const Node*> fs;
    flatten_product(n, &fs);
    if (fs.size() == 1) return as_dft(fs[0], f, err);
    if (fs.size() >= 7) {
        std::string pe;
        if (as_pease(fs, f, &pe)) return true;
        return *err = "not a DFT: Eq. 2 has four factors (or their transpose); " + pe, false;
    }
    if (fs.size() != 4)
        return *err = "not a DFT: Eq. 2 has four factors (DFT_K (x) I_M) . twiddle(N,M) . (I_K (x) DFT_M) . "
                      "Permute(N,K) (or their transpose)",
               false;
    const Node *f1 = fs[0], *f2 = fs[1], *f3 = fs[2], *f4 = fs[3];
    if (f1->kind == kPermute) return as_dft_transposed(fs, f, err);
    if (f1->kind != kKron || f1->r->kind != kIdent)
        return *err = "first factor must be (DFT_K (x) I_M)", false;
    if (f3->kind != kKron || f3->l->kind != kIdent) return *err = "third factor must be (I_K (x) DFT_M)", false;
    if (f2->kind != kTwiddle) return *err = "second factor must be twiddle(N, M)", false;
    if (f4->kind != kPermute) return *err = "fourth factor must be Permute(N, K)", false;
    DftForm x, y;
    if (!as_dft(f1->l.get(), &x, err) || !as_dft(f3->r.get(), &y, err)) return false;
    const int64_t K = x.n, M = y.n, N = K * M;
    if (f1->r->a != M) return *err = "first factor: I_M must match DFT_M of the third factor", false;
    if (f3->l->a != K) return *err = "third factor: I_K must match DFT_K of the first factor", false;
    if (f2->a != N || f2->b != M) return *err = "second factor must be twiddle(N, M) with N = K*M", false;
    if (f4->a != N || f4->b != K) return *err = "fourth factor must be Permute(N, K) with N = K*M", false;
    f->n = N;
    f->k_top = K;
    f->bare = x.k_top == 0 && y.k_top == 0;
    f->leaves = y.leaves;  // DFT_M runs first (after the permutation), then DFT_K
    f->leaves.insert(f->leaves.end(), x.leaves.begin(), x.leaves.end());
    return true;
}

gbfft_status check(const char* text, DftForm* f, std::string* err) {
    if (!text) return *err = "null formula", GBFFT_ERR_INVALID_ARG;
    Parser p(text);
    auto root = p.program();
    if (!root) return *err = p.err, GBFFT_ERR_INVALID_ARG;
    // Strip a trailing input vector: <formula> · InputComplex.
    const Node* body = root.get();
    if (body->kind == kInput) return *err = "the formula has no operator", GBFFT_ERR_INVALID_ARG;
    std::unique_ptr<Node> owned;
    if (body->kind == kProd) {
        // find the rightmost factor of the top-level product chain
        Node* parent = nullptr;
        Node* cur = root.get();
        while (cur->kind == kProd && cur->r->kind == kProd) {
            parent = cur;
            cur = cur->r.get();
        }
        if (cur->kind == kProd && cur->r->kind == kInput) {
            if (parent) {
                parent->r = std::move(cur->l);
            } else {
                owned = std::move(root->l);
                body = owned.get();
            }
        }
    }
    if (!dim(body, err)) return GBFFT_ERR_INVALID_ARG;
    if (!as_dft(body, f, err)) return GBFFT_ERR_INVALID_ARG;
    return GBFFT_OK;
}

void put_err(const std::string& e, char* buf, size_t len) {
    if (!buf || len == 0) return;
    std::snprintf(buf, len, "%s", e.c_str());
}

}  // namespace

bool formula_plan_choice(const char* text, int64_t* n, std::vector<int64_t>* leaves, int64_t* k_top, bool* bare,
                         bool* pease) {
    DftForm f;
    std::string err;
    if (check(text, &f, &err) != GBFFT_OK) return false;
    *n = f.n;
    *leaves = f.leaves;
    *k_top = f.k_top;
    *bare = f.bare;
    *pease = f.pease;
    return true;
}

}  // namespace gbfft

using namespace gbfft;

extern "C" {

gbfft_status gbfft_formula_check(const char* formula, int64_t* n, int* leaves, int max_leaves, int* nleaves,
                                 int64_t* k_outer, char* err, size_t err_len) {
    DftForm f;
    std::string e;
    const gbfft_status st = check(formula, &f, &e);
    if (st != GBFFT_OK) {
        put_err(e, err, err_len);
        return st;
    }
    put_err("", err, err_len);
    if (n) *n = f.n;
    if (k_outer) *k_outer = f.k_top;
    if (nleaves) *nleaves = (int)f.leaves.size();
    if (leaves)
        for (int i = 0; i < (int)f.leaves.size() && i < max_leaves; ++i) leaves[i] = (int)f.leaves[i];
    return GBFFT_OK;
}

int gbfft_formula_form(const char* formula) {
    DftForm f;
    std::string e;
    if (check(formula, &f, &e) != GBFFT_OK) return -1;
    return f.pease ? 2 : (f.transposed ? 1 : 0);
}

}  // extern "C"
