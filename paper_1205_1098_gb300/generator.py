"""Generator of fused passes for BLAS-1/2 sequences given as a short program.

The paper's compiler takes a kernel written as linear-algebra statements
over declared matrices, vectors and scalars (its input language, Section II
and Fig. 1), builds the dataflow graph, and fuses the loops of operations
that share an operand, where the dependences allow it (Section III-C: a
vector formed by a reduction is not available until the reduction is
complete, so its consumers cannot share the loop that forms it).  This
module does the same for the GPU panel engine of this library:

  * the statements are parsed and rewritten as linear combinations of
    matrix-vector products, vectors and rank-one updates (nested products
    become temporaries, as the paper's dataflow graph names them);
  * every product is a node of the matrix it reads; the nodes whose input
    vectors are complete are grouped into passes that read each matrix once:
    a transposed and a non-transposed product of the same matrix share a
    pass (mode QS), products of two equally shaped matrices with the same
    input vector share one (Q2), and a rank-update that forms a matrix
    shares its pass with one product of the formed matrix (G1, G1Q);
  * a vector is complete after the combine that adds its pass partials, so a
    product that consumes it goes to a later pass (the reduction rule);
  * a row-major matrix (declared `matrix(row)`) is used as its column-major
    transpose, the two products exchanging roles.

The result is a program of bto_instr records (include/bto.h) that the
native runtime (bto_program_run) executes.

Input language (an optional title line, then declarations and statements,
one per line, `#` comments):

    GEMVER
    in:  A : matrix, u1 v1 u2 v2 y z : vector, alpha beta : scalar
    out: B : matrix, x w : vector
    B = A + u1 * v1' + u2 * v2'
    x = beta * B' * y + z
    w = alpha * B * x

Types: `matrix`, `matrix(row)`, `matrix(column)`, `vector`, `vector(column)`,
`scalar`.  Targets that are not declared are temporaries.  Every name is
assigned once, inputs never.  Matrix statements have the form
`M = N + u * v' [+ ...]` with one or two rank-one terms.  Dot products
(`x' * y`) are outside this generator (AXPYDOT has its own kernel).
"""
import re

from . import _lib as L


class SpecError(ValueError):
    """A program the generator cannot read or cannot plan."""


# ------------------------------------------------------------------ parsing

_TOKEN = re.compile(r"\s*(?:(\d+\.\d*(?:[eE][-+]?\d+)?|\.\d+(?:[eE][-+]?\d+)?|\d+(?:[eE][-+]?\d+)?)|"
                    r"([A-Za-z_][A-Za-z_0-9]*)|(.))")


def _tokens(text):
    out = []
    for num, name, op in _TOKEN.findall(text):
        if num:
            out.append(("num", float(num)))
        elif name:
            out.append(("name", name))
        elif op.strip():
            if op not in "+-*()'":
                raise SpecError("unexpected character %r in %r" % (op, text))
            out.append(("op", op))
    return out


class _Parser:
    """Recursive descent over  expr := term (('+'|'-') term)* ;
    term := unary ('*' unary)* ; unary := '-' unary | post ;
    post := prim "'"* ; prim := NAME | NUMBER | '(' expr ')'."""

    def __init__(self, toks):
        self.t, self.i = toks, 0

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else (None, None)

    def take(self, kind=None, val=None):
        k, v = self.peek()
        if k is None or (kind and k != kind) or (val is not None and v != val):
            raise SpecError("expected %s near token %d" % (val or kind, self.i))
        self.i += 1
        return v

    def parse(self):
        e = self.expr()
        if self.i != len(self.t):
            raise SpecError("trailing tokens in expression")
        return e

    def expr(self):
        e = self.term()
        while self.peek() in (("op", "+"), ("op", "-")):
            op = self.take()
            e = ("add" if op == "+" else "sub", e, self.term())
        return e

    def term(self):
        e = self.unary()
        while self.peek() == ("op", "*"):
            self.take()
            e = ("mul", e, self.unary())
        return e

    def unary(self):
        if self.peek() == ("op", "-"):
            self.take()
            return ("neg", self.unary())
        return self.post()

    def post(self):
        e = self.prim()
        while self.peek() == ("op", "'"):
            self.take()
            e = ("tr", e)
        return e

    def prim(self):
        k, v = self.peek()
        if k == "num":
            self.take()
            return ("num", v)
        if k == "name":
            self.take()
            return ("name", v)
        if (k, v) == ("op", "("):
            self.take()
            e = self.expr()
            self.take("op", ")")
            return e
        raise SpecError("unexpected token %r" % (v,))


_TYPES = {"matrix": ("matrix", "col"), "matrix(column)": ("matrix", "col"), "matrix(col)": ("matrix", "col"),
          "matrix(row)": ("matrix", "row"), "vector": ("vector", None), "vector(column)": ("vector", None),
          "scalar": ("scalar", None)}


class Spec:
    """A parsed program: name, declarations {name: (kind, orient, io)} and
    statements [(target, ast)] in order."""

    def __init__(self, name, decls, stmts):
        self.name, self.decls, self.stmts = name, decls, stmts


def parse(text):
    name, decls, stmts, section = None, {}, [], None
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].strip()
        if not line or line in ("{", "}"):
            continue
        line = line.strip("{}").strip()
        low = line.lower()
        if low.startswith("in:") or low.startswith("out:"):
            section = "in" if low.startswith("in:") else "out"
            line = line.split(":", 1)[1].strip()
            if not line:
                continue
        if "=" in line:
            section = None
            tgt, rhs = line.split("=", 1)
            tgt = tgt.strip()
            if not re.fullmatch(r"[A-Za-z_][A-Za-z_0-9]*", tgt):
                raise SpecError("bad assignment target %r" % tgt)
            stmts.append((tgt, _Parser(_tokens(rhs)).parse()))
            continue
        if section is None:
            if name is None and not decls:
                name = line          # the title line
                continue
            raise SpecError("line outside a declaration or statement: %r" % raw)
        for entry in line.split(","):
            entry = entry.strip()
            if not entry:
                continue
            if ":" not in entry:
                raise SpecError("declaration without a type: %r" % entry)
            names, ty = entry.split(":", 1)
            ty = ty.replace(" ", "").lower()
            if ty not in _TYPES:
                raise SpecError("unknown type %r" % ty)
            kind, orient = _TYPES[ty]
            for n in names.split():
                if n in decls:
                    raise SpecError("%s declared twice" % n)
                decls[n] = (kind, orient, section)
    if not stmts:
        raise SpecError("no statements")
    return Spec(name or "sequence", decls, stmts)


# ------------------------------------------------------------------ normal form
#
# Scalars are coefficient lists: a product of names and numbers.  A vector
# value is a list of terms (coef, atom), atom = ("v", name) or
# ("mv", matrix, transposed, name).  A matrix value is a list of terms
# ("mat", coef, name, transposed) or ("outer", coef, u, v).


class _S:
    def __init__(self, f):
        self.f = list(f)


class _V:
    def __init__(self, terms):
        self.terms = list(terms)


class _RV:            # a transposed vector (only inside u * v')
    def __init__(self, name):
        self.name = name


class _M:
    def __init__(self, terms):
        self.terms = list(terms)


class _Normaliser:
    def __init__(self, decls):
        self.decls = decls
        self.kinds = {n: d[0] for n, d in decls.items()}
        self.temps = []          # (name, _V) statements created on the way
        self.ntemp = 0

    def temp_of(self, v):
        """A vector name holding the value v (a new temporary unless v is a plain name)."""
        if len(v.terms) == 1 and v.terms[0][1][0] == "v" and v.terms[0][0] == [1.0]:
            return v.terms[0][1][1]
        self.ntemp += 1
        name = "_t%d" % self.ntemp
        self.temps.append((name, v))
        self.kinds[name] = "vector"
        return name

    def norm(self, e):
        k = e[0]
        if k == "num":
            return _S([e[1]])
        if k == "name":
            n = e[1]
            if n not in self.kinds:
                raise SpecError("%s is not declared or assigned before use" % n)
            kind = self.kinds[n]
            if kind == "scalar":
                return _S([n])
            if kind == "vector":
                return _V([([1.0], ("v", n))])
            return _M([("mat", [1.0], n, False)])
        if k == "neg":
            return self.scale(_S([-1.0]), self.norm(e[1]))
        if k == "tr":
            x = self.norm(e[1])
            if isinstance(x, _S):
                return x
            if isinstance(x, _V):
                if len(x.terms) == 1 and x.terms[0][1][0] == "v" and x.terms[0][0] == [1.0]:
                    return _RV(x.terms[0][1][1])
                raise SpecError("only a named vector can be transposed")
            if isinstance(x, _RV):
                return _V([([1.0], ("v", x.name))])
            if len(x.terms) == 1 and x.terms[0][0] == "mat":
                _, c, n, t = x.terms[0]
                return _M([("mat", c, n, not t)])
            raise SpecError("only a named matrix can be transposed")
        if k in ("add", "sub"):
            a, b = self.norm(e[1]), self.norm(e[2])
            if k == "sub":
                b = self.scale(_S([-1.0]), b)
            if isinstance(a, _V) and isinstance(b, _V):
                return _V(a.terms + b.terms)
            if isinstance(a, _M) and isinstance(b, _M):
                return _M(a.terms + b.terms)
            raise SpecError("cannot add these operands (scalar sums, or a vector and a matrix)")
        if k == "mul":
            return self.mul(self.norm(e[1]), self.norm(e[2]))
        raise SpecError("bad expression")

    def scale(self, s, x):
        if isinstance(x, _S):
            return _S(s.f + x.f)
        if isinstance(x, _V):
            return _V([(s.f + c, a) for c, a in x.terms])
        if isinstance(x, _M):
            out = []
            for t in x.terms:
                out.append((t[0], s.f + t[1]) + tuple(t[2:]))
            return _M(out)
        raise SpecError("cannot scale a transposed vector")

    def mul(self, a, b):
        if isinstance(a, _S):
            return self.scale(a, b)
        if isinstance(b, _S):
            return self.scale(b, a)
        if isinstance(a, _M) and isinstance(b, _V):
            if len(a.terms) != 1 or a.terms[0][0] != "mat":
                raise SpecError("a product needs a single (possibly scaled or transposed) matrix")
            _, c, mname, tr = a.terms[0]
            if len(b.terms) == 1 and b.terms[0][1][0] == "v":
                coef, (_, vname) = b.terms[0]
                return _V([(c + coef, ("mv", mname, tr, vname))])
            return _V([(c, ("mv", mname, tr, self.temp_of(b)))])
        if isinstance(a, _V) and isinstance(b, _RV):
            if len(a.terms) != 1 or a.terms[0][1][0] != "v":
                raise SpecError("a rank-one term needs a named vector on the left")
            coef, (_, u) = a.terms[0]
            return _M([("outer", coef, u, b.name)])
        if isinstance(a, _RV) and isinstance(b, _V):
            raise SpecError("dot products (x' * y) are outside the generator")
        if isinstance(a, _M) and isinstance(b, _M):
            raise SpecError("matrix-matrix products are outside the generator")
        raise SpecError("unsupported product")


# ------------------------------------------------------------------ dimensions


class _Dims:
    """Union-find over dimension symbols: ('rows', M), ('cols', M), ('len', v)."""

    def __init__(self):
        self.parent = {}

    def find(self, x):
        self.parent.setdefault(x, x)
        while self.parent[x] != x:
            self.parent[x] = self.parent[self.parent[x]]
            x = self.parent[x]
        return x

    def union(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra != rb:
            self.parent[ra] = rb


# ------------------------------------------------------------------ planning


class Plan:
    """A planned program: `steps` (symbolic passes, combines and WAXPBY steps)
    and `passes` (short descriptions, for inspection and tests)."""

    def __init__(self, spec, steps, temps, dims, orient, decls, matrix_outs):
        self.spec, self.steps, self.temps, self.dims = spec, steps, temps, dims
        self.orient, self.decls, self.matrix_outs = orient, decls, matrix_outs

    @property
    def passes(self):
        return [s for s in self.steps if s["op"] == "pass"]

    def describe(self):
        lines = []
        for s in self.steps:
            if s["op"] == "pass":
                prods = ", ".join("%s <- %s" % (k, v) for k, v in s["forms"])
                lines.append("pass %-4s over %s%s: %s" % (s["mode"], s["A"] + ("" if s["B"] is None else
                                                                                 " and " + s["B"]),
                                                            " (reversed)" if s["reverse"] else "", prods))
            elif s["op"] == "combine":
                lines.append("combine -> %s" % s["out"])
            else:
                lines.append("waxpby -> %s" % s["out"])
        return "\n".join(lines)

    # -------------------------------------------------------------- running

    def vector_length(self, name, shapes):
        root = self.dims.find(("len", name))
        for mname, (r, c) in shapes.items():
            if self.dims.find(("rows", mname)) == root:
                return int(r)
            if self.dims.find(("cols", mname)) == root:
                return int(c)
        return None

    def _shapes(self, shapes):
        out = dict(shapes)
        for b, a in self.matrix_outs.items():
            if b not in out:
                if a not in out:
                    raise SpecError("shape of %s is needed" % a)
                out[b] = out[a]
        for n, d in self.decls.items():
            if d[0] == "matrix" and n not in out:
                raise SpecError("shape of matrix %s is needed" % n)
        # Every dimension the program ties together must have one size.
        size = {}
        for mname, (r, c) in out.items():
            for key, v in ((("rows", mname), r), (("cols", mname), c)):
                root = self.dims.find(key)
                if size.setdefault(root, int(v)) != int(v):
                    raise SpecError("shapes disagree: %s of %s is %d, tied to a dimension of size %d"
                                    % (key[0], mname, v, size[root]))
        return out

    def program(self, bindings, shapes, lds=None, device="cuda"):
        """(ctypes Instr array, temporaries kept alive) for
        the given device buffers (torch tensors), scalars (floats) and matrix
        shapes {name: (rows, cols)} (lds: leading dimensions, default the
        stored row count)."""
        import torch
        shapes = self._shapes(shapes)
        lds = dict(lds or {})
        keep = {}
        buf = dict(bindings)
        lens = {}

        def vlen(name):
            if name not in lens:
                n = self.vector_length(name, shapes)
                if n is None:
                    t = buf.get(name)
                    if t is None:
                        raise SpecError("length of vector %s is not fixed by a matrix" % name)
                    n = t.numel()
                lens[name] = n
            return lens[name]

        for n, d in self.decls.items():
            if d[2] in ("in", "out") and d[0] != "scalar" and n not in buf:
                raise SpecError("no buffer bound to %s" % n)
            if d[0] == "scalar" and not isinstance(bindings.get(n), (int, float)):
                raise SpecError("scalar %s needs a number" % n)
        for n, t in bindings.items():
            if n in self.decls and self.decls[n][0] != "scalar":
                if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous():
                    raise SpecError("%s must be a contiguous float64 tensor" % n)
                if t.device.type != torch.device(device).type:
                    raise SpecError("%s is on %s, the program runs on %s" % (n, t.device, device))
        for t in self.temps:
            buf[t] = keep[t] = torch.empty(max(vlen(t), 1), dtype=torch.float64, device=device)
        for n, d in self.decls.items():
            if d[0] == "vector" and buf[n].numel() < vlen(n):
                raise SpecError("vector %s has %d elements, needs %d" % (n, buf[n].numel(), vlen(n)))

        def stored(mname):
            r, c = shapes[mname]
            return (r, c) if self.orient[mname] == "col" else (c, r)

        def ld_of(mname):
            if mname in lds:
                return int(lds[mname])
            return max(1, stored(mname)[0])

        for mname in shapes:
            if mname in buf:
                sm, sn = stored(mname)
                need = (sn - 1) * ld_of(mname) + sm if sm and sn else 0
                if buf[mname].numel() < need:
                    raise SpecError("matrix %s has %d elements, needs %d" % (mname, buf[mname].numel(), need))

        def coef(f):
            v = 1.0
            for x in f:
                v *= float(x) if isinstance(x, float) else float(bindings[x])
            return v

        def ptr(name):
            if name is None:
                return None
            t = buf[name]
            return t.data_ptr() if t.numel() else None

        prog = (L.Instr * len(self.steps))()
        for i, s in enumerate(self.steps):
            I = prog[i]
            I.slot_q = I.slot_q2 = I.slot_s = I.src1 = I.src2 = -1
            if s["op"] == "pass":
                I.op = L.BTO_INSTR_PASS
                I.mode = getattr(L, "BTO_PASS_" + s["mode"])
                I.reverse = 1 if s["reverse"] else 0
                sm, sn = stored(s["A"])
                I.m, I.n = sm, sn
                I.A, I.lda = ptr(s["A"]), ld_of(s["A"])
                if s["B"] is not None:
                    I.B, I.ldb = ptr(s["B"]), ld_of(s["B"])
                if s["Bout"] is not None:
                    I.Bout, I.ldbo = ptr(s["Bout"]), ld_of(s["Bout"])
                for f in ("p", "r", "u1", "v1", "u2", "v2"):
                    if s.get(f) is not None:
                        setattr(I, f, ptr(s[f]))
                for f in ("slot_q", "slot_q2", "slot_s"):
                    if s.get(f) is not None:
                        setattr(I, f, s[f])
            elif s["op"] == "combine":
                I.op = L.BTO_INSTR_COMBINE
                I.n = vlen(s["out"])
                I.out = ptr(s["out"])
                if s["src1"] is not None:
                    I.src1, I.a1 = s["src1"][1], coef(s["src1"][0])
                if s["src2"] is not None:
                    I.src2, I.a2 = s["src2"][1], coef(s["src2"][0])
                if s["x"] is not None:
                    I.x, I.b = ptr(s["x"][1]), coef(s["x"][0])
            else:
                I.op = L.BTO_INSTR_WAXPBY
                I.n = vlen(s["out"])
                I.out = ptr(s["out"])
                I.x, I.a1 = ptr(s["x"][1]), coef(s["x"][0])
                I.y, I.b = ptr(s["y"][1]), coef(s["y"][0])
        return prog, keep

    def run(self, bindings, shapes, lds=None, stream=None):
        """Runs the program on the current device (enqueued on `stream`)."""
        import torch
        prog, keep = self.program(bindings, shapes, lds)
        st, bad = L.bto_program_check(prog)
        if st != L.BTO_OK:
            raise SpecError("program check failed at instruction %d" % bad)
        nb = L.bto_program_workspace_bytes(prog)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
        L.bto_program_run(prog, ws, nb, stream)
        keep["_ws"] = ws
        return keep


MAX_FUSE = {"qs": True, "q2": True, "update": True}


def compile(text, policy=None):
    """Parses and plans a program (see the module docstring).  `policy`
    chooses which fusions the planner may make (all of them by default, the
    paper's Max-Fuse starting point): "qs" pairs a non-transposed and a
    transposed product of one matrix in a pass, "q2" pairs products of two
    matrices on one input, "update" lets a pass that forms a matrix also form
    a product of it."""
    spec = parse(text)
    decls = spec.decls
    norm = _Normaliser(decls)
    stmts = []            # ("vec", target, _V) or ("mat", target, base, [(coef, u, v)])
    assigned = set()
    orient = {n: d[1] for n, d in decls.items() if d[0] == "matrix"}
    matrix_outs = {}
    for tgt, ast in spec.stmts:
        if tgt in decls and decls[tgt][2] == "in":
            raise SpecError("%s is an input and cannot be assigned" % tgt)
        if tgt in assigned:
            raise SpecError("%s is assigned twice" % tgt)
        val = norm.norm(ast)
        new_temps, norm.temps = norm.temps, []
        for tn, tv in new_temps:
            stmts.append(("vec", tn, tv))
        if isinstance(val, _V):
            if tgt in decls and decls[tgt][0] != "vector":
                raise SpecError("%s is declared %s but assigned a vector" % (tgt, decls[tgt][0]))
            stmts.append(("vec", tgt, val))
            norm.kinds[tgt] = "vector"
        elif isinstance(val, _M):
            if tgt in decls and decls[tgt][0] != "matrix":
                raise SpecError("%s is declared %s but assigned a matrix" % (tgt, decls[tgt][0]))
            mats = [t for t in val.terms if t[0] == "mat"]
            outs = [t for t in val.terms if t[0] == "outer"]
            if len(mats) != 1 or mats[0][3] or any(not isinstance(x, float) for x in mats[0][1]) or \
                    _prod(mats[0][1]) != 1.0:
                raise SpecError("a matrix statement is M = N + u * v' (+ u2 * v2') with N unscaled")
            if not 1 <= len(outs) <= 2:
                raise SpecError("a matrix statement takes one or two rank-one terms")
            base = mats[0][2]
            o = orient.get(base, "col")
            if tgt in decls and decls[tgt][1] != o:
                raise SpecError("%s must have the storage order of %s" % (tgt, base))
            orient[tgt] = o
            matrix_outs[tgt] = base
            stmts.append(("mat", tgt, base, [(c, u, v) for _, c, u, v in outs]))
            norm.kinds[tgt] = "matrix"
        else:
            raise SpecError("%s must be assigned a vector or a matrix" % tgt)
        assigned.add(tgt)
    for n, d in decls.items():
        if d[2] == "out" and n not in assigned:
            raise SpecError("output %s is never assigned" % n)
    return _plan(spec, stmts, orient, matrix_outs, dict(MAX_FUSE, **(policy or {})))


def fusion_choices(text):
    """Every distinct plan the fusion policies give for a program, as
    [(policy, Plan)], Max-Fuse first: the legal points among which a
    measured search (`search`) chooses, as the paper's search does."""
    out, seen = [], set()
    for qs in (True, False):
        for q2 in (True, False):
            for update in (True, False):
                pol = {"qs": qs, "q2": q2, "update": update}
                P = compile(text, pol)
                key = P.describe()
                if key not in seen:
                    seen.add(key)
                    out.append((pol, P))
    return out


def search(text, bindings, shapes, lds=None, reps=5):
    """Measures every distinct fusion choice of a program on the current
    device (median of `reps` calls after 2 warm-ups, CUDA events) and returns
    {"best": policy, "best_ms": ms, "table": [(policy, passes, ms)]}."""
    import torch
    table = []
    st = torch.cuda.current_stream()
    for pol, P in fusion_choices(text):
        prog, keep = P.program(bindings, shapes, lds)
        nb = L.bto_program_workspace_bytes(prog)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            L.bto_program_run(prog, ws, nb, None)
        evs = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            L.bto_program_run(prog, ws, nb, None)
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sorted(a.elapsed_time(b) for a, b in evs)[reps // 2]
        table.append((pol, [x["mode"] for x in P.passes], ms))
        del ws, keep
    best = min(table, key=lambda t: t[2])
    return {"best": best[0], "best_ms": best[2], "table": table}


def _prod(f):
    v = 1.0
    for x in f:
        v *= x
    return v


def _plan(spec, stmts, orient, matrix_outs, policy):
    return _Planner(spec, stmts, orient, matrix_outs, policy).plan()


class _Planner:
    """Schedules a normalised program into passes of the engine, level by
    level: a level forms every product whose input vector is complete, then
    emits the combines that complete vectors (the reduction rule)."""

    def __init__(self, spec, stmts, orient, matrix_outs, policy):
        self.spec, self.decls, self.orient = spec, spec.decls, orient
        self.matrix_outs, self.policy = matrix_outs, policy
        self.dims = _Dims()
        self.temps = [s[1] for s in stmts if s[1] not in self.decls]
        self.nz = 0                  # numbering of the scaled and zero temporaries
        self.nw = 0                  # numbering of the WAXPBY temporaries
        self.steps = []
        self.nslots = 0
        self.last = (None, False)    # matrix of the previous pass, and whether it ran reversed
        stmts = self._expand_updates(stmts)
        self._tie_vector_lengths(stmts)
        self._collect(stmts)

    # ---------------------------------------------------------- preparation

    def _temp(self, prefix, dim):
        self.nz += 1
        name = "%s%d" % (prefix, self.nz)
        self.temps.append(name)
        self.dims.union(("len", name), dim)
        return name

    def _expand_updates(self, stmts):
        """Rank-one coefficients other than 1 become scaled temporaries; a
        single rank-one term gets a zero second term (the engine's update
        adds two)."""
        out = []
        for st in stmts:
            if st[0] != "mat":
                out.append(st)
                continue
            _, tgt, base, outs = st
            pairs = []
            for c, u, v in outs:
                if any(isinstance(x, str) for x in c) or _prod(c) != 1.0:
                    su = self._temp("_s", ("len", u))
                    out.append(("vec", su, _V([(c, ("v", u))])))
                    u = su
                pairs.append((u, v))
            self.dims.union(("rows", tgt), ("rows", base))
            self.dims.union(("cols", tgt), ("cols", base))
            for u, v in pairs:
                self.dims.union(("len", u), ("rows", base))
                self.dims.union(("len", v), ("cols", base))
            if len(pairs) == 1:
                zu, zv = self._temp("_z", ("rows", base)), self._temp("_z", ("cols", base))
                out.append(("vec", zu, _V([])))          # a statement with no terms: zeros
                out.append(("vec", zv, _V([])))
                pairs.append((zu, zv))
            out.append(("mat", tgt, base, pairs))
        return out

    def _tie_vector_lengths(self, stmts):
        for st in stmts:
            if st[0] != "vec":
                continue
            tgt = st[1]
            for c, a in st[2].terms:
                if a[0] == "v":
                    self.dims.union(("len", tgt), ("len", a[1]))
                else:
                    _, M, tr, x = a
                    self.dims.union(("len", x), ("rows" if tr else "cols", M))
                    self.dims.union(("len", tgt), ("cols" if tr else "rows", M))

    def _stored_kind(self, M, tr):
        # Column-major: M x is the row accumulators (q), M' y the column sums (s).
        q = not tr
        return "q" if (q if self.orient[M] == "col" else not q) else "s"

    def _collect(self, stmts):
        """Product nodes, vector statements (as combines of nodes and
        vectors) and rank updates."""
        self.nodes, self.vec_stmts, self.upd = [], [], []
        for st in stmts:
            if st[0] == "vec":
                terms = []
                for c, a in st[2].terms:
                    if a[0] == "mv":
                        node = {"id": len(self.nodes), "M": a[1], "tr": a[2], "kind": self._stored_kind(a[1], a[2]),
                                "x": a[3], "done": False, "slot": None}
                        self.nodes.append(node)
                        terms.append((c, ("node", node["id"])))
                    else:
                        terms.append((c, a))
                self.vec_stmts.append({"out": st[1], "terms": terms, "done": False})
            else:
                self.upd.append({"out": st[1], "base": st[2], "pairs": st[3], "done": False})

    # ---------------------------------------------------------- steps

    def _new_slot(self):
        s = self.nslots
        self.nslots += 1
        if s >= L.BTO_PROGRAM_MAX_SLOTS:
            raise SpecError("program needs more than %d partial slots" % L.BTO_PROGRAM_MAX_SLOTS)
        return s

    def _add_pass(self, mode, A, forms, B=None, Bout=None, p=None, r=None, upd_vecs=None, nq=None, nq2=None,
                  ns=None):
        # A pass over the matrix the previous pass read or wrote runs its
        # tiles in reverse, so the tail still in L2 is read first.
        rev = (self.last[0] is not None and self.last[0] in (A, Bout)) and not self.last[1]
        s = {"op": "pass", "mode": mode, "A": A, "B": B, "Bout": Bout, "p": p, "r": r, "reverse": rev,
             "forms": forms, "slot_q": None, "slot_q2": None, "slot_s": None}
        if upd_vecs:
            s.update(upd_vecs)
        for key, nd in (("slot_q", nq), ("slot_q2", nq2), ("slot_s", ns)):
            if nd is not None:
                nd["slot"] = s[key] = self._new_slot()
        self.steps.append(s)
        self.last = (Bout or A, rev)
        for nd in (nq, nq2, ns):
            if nd is not None:
                nd["done"] = True

    @staticmethod
    def _label(nd):
        # The product as the program writes it; a pass that forms a matrix
        # with no product of it ready sums a zero vector.
        if nd["id"] < 0:
            return "(no product)"
        return "%s%s %s" % (nd["M"], "'" if nd["tr"] else "", nd["x"])

    def _emit_combines(self, vs):
        """out = sum of scaled slot sums and scaled vectors: vector terms
        beyond the first are folded with WAXPBY first, then combines add two
        slots at a time (the later ones onto out itself)."""
        out = vs["out"]
        parts = [(c, self.nodes[a[1]]["slot"]) for c, a in vs["terms"] if a[0] == "node"]
        vecs = [(c, a[1]) for c, a in vs["terms"] if a[0] == "v"]
        if len(vecs) >= 2:
            cur = vecs[0]
            for k, nxt in enumerate(vecs[1:]):
                if k == len(vecs) - 2 and not parts:
                    dst = out
                else:
                    self.nw += 1
                    dst = "_w%d" % self.nw
                    self.temps.append(dst)
                    self.dims.union(("len", dst), ("len", out))
                self.steps.append({"op": "waxpby", "out": dst, "x": cur, "y": nxt})
                cur = ([1.0], dst)
            if not parts:
                return
            vecs = [cur]
        x = vecs[0] if vecs else None
        if not parts:
            self.steps.append({"op": "combine", "out": out, "src1": None, "src2": None, "x": x})
            return
        first = True
        while parts:
            p1 = parts.pop(0)
            p2 = parts.pop(0) if parts else None
            self.steps.append({"op": "combine", "out": out, "src1": p1, "src2": p2,
                               "x": x if first else ([1.0], out)})
            first = False

    # ---------------------------------------------------------- levels

    def _update_passes(self, ready_upd, ready):
        """Each ready update forms its matrix in a pass that also forms one
        ready product of that matrix (G1 for a column sum, G1Q for a row
        product), or a column sum of zeros when none is ready."""
        for u in ready_upd:
            mine = [nd for nd in ready if nd["M"] == u["out"]] if self.policy["update"] else []
            s_nodes = [nd for nd in mine if nd["kind"] == "s"]
            q_nodes = [nd for nd in mine if nd["kind"] == "q"]
            (a1, b1), (a2, b2) = u["pairs"]
            if self.orient[u["out"]] == "row":        # stored transpose: u and v exchange roles
                vecs = {"u1": b1, "v1": a1, "u2": b2, "v2": a2}
            else:
                vecs = {"u1": a1, "v1": b1, "u2": a2, "v2": b2}
            if s_nodes or not q_nodes:
                nd = s_nodes[0] if s_nodes else None
                if nd is None:
                    z = self._temp("_z", ("rows" if self.orient[u["out"]] == "col" else "cols", u["base"]))
                    nd = {"id": -1, "M": u["out"], "kind": "s", "x": z, "done": False, "slot": None}
                    self.steps.append({"op": "combine", "out": z, "src1": None, "src2": None, "x": None})
                self._add_pass("G1", u["base"], [("s", self._label(nd))], Bout=u["out"], r=nd["x"], upd_vecs=vecs,
                               ns=nd)
            else:
                nd = q_nodes[0]
                self._add_pass("G1Q", u["base"], [("q", self._label(nd))], Bout=u["out"], p=nd["x"],
                               upd_vecs=vecs, nq=nd)
            u["done"] = True
        return bool(ready_upd)

    def _q2_mate(self, nq, singles_q):
        if not self.policy["q2"]:
            return None
        f = self.dims.find
        for cand in singles_q:
            if cand["x"] == nq["x"] and cand["M"] != nq["M"] and self.orient[cand["M"]] == self.orient[nq["M"]] and \
                    f(("rows", cand["M"])) == f(("rows", nq["M"])) and f(("cols", cand["M"])) == f(("cols", nq["M"])):
                return cand
        return None

    def _plain_passes(self, ready, avail):
        """Products of available matrices: a row and a column product of one
        matrix share a QS pass, row products of two equally shaped matrices
        on one input a Q2 pass; the rest take a pass each."""
        progress = False
        by_m = {}
        for nd in ready:
            if not nd["done"] and nd["M"] in avail:
                by_m.setdefault(nd["M"], []).append(nd)
        singles_q = []
        for M, lst in by_m.items():
            qs = [nd for nd in lst if nd["kind"] == "q"]
            ss = [nd for nd in lst if nd["kind"] == "s"]
            while qs and ss and self.policy["qs"]:
                nq, ns = qs.pop(0), ss.pop(0)
                self._add_pass("QS", M, [("q", self._label(nq)), ("s", self._label(ns))], p=nq["x"], r=ns["x"],
                               nq=nq, ns=ns)
                progress = True
            for ns in ss:
                self._add_pass("S", M, [("s", self._label(ns))], r=ns["x"], ns=ns)
                progress = True
            singles_q.extend(qs)
        while singles_q:
            nq = singles_q.pop(0)
            mate = self._q2_mate(nq, singles_q)
            if mate is not None:
                singles_q.remove(mate)
                self._add_pass("Q2", nq["M"], [("q", self._label(nq)), ("q2", self._label(mate))], B=mate["M"],
                               p=nq["x"], nq=nq, nq2=mate)
            else:
                self._add_pass("Q", nq["M"], [("q", self._label(nq))], p=nq["x"], nq=nq)
            progress = True
        return progress

    def _complete_vectors(self, avail):
        """Combines of every statement whose products are complete, in order;
        a completed vector may complete a later statement at once."""
        progress, changed = False, True
        while changed:
            changed = False
            for vs in self.vec_stmts:
                if vs["done"]:
                    continue
                if all(self.nodes[a[1]]["done"] if a[0] == "node" else a[1] in avail for c, a in vs["terms"]):
                    self._emit_combines(vs)
                    vs["done"] = True
                    avail.add(vs["out"])
                    changed = progress = True
        return progress

    def plan(self):
        avail = {n for n, d in self.decls.items() if d[2] == "in"}
        while True:
            pending_nodes = [nd for nd in self.nodes if not nd["done"]]
            pending_upd = [u for u in self.upd if not u["done"]]
            if not pending_nodes and not pending_upd and all(v["done"] for v in self.vec_stmts):
                break
            ready_upd = [u for u in pending_upd
                         if u["base"] in avail and all(a in avail and b in avail for a, b in u["pairs"])]
            forming = {u["out"] for u in ready_upd}
            ready = [nd for nd in pending_nodes if nd["x"] in avail and (nd["M"] in avail or nd["M"] in forming)]
            progress = self._update_passes(ready_upd, ready)
            progress |= self._plain_passes(ready, avail)
            for u in self.upd:
                if u["done"]:
                    avail.add(u["out"])
            progress |= self._complete_vectors(avail)
            if not progress:
                raise SpecError("cannot schedule the remaining statements (a value is used before it is formed)")
        return Plan(self.spec, self.steps, list(dict.fromkeys(self.temps)), self.dims, self.orient, self.decls,
                    self.matrix_outs)
