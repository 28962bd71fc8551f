"""Host logic of the functional entry points (no GPU): lattice extents read from
the link tensor, one context per (device, extents, mass, boundary), links staged
again after an in-place change or for a different tensor."""
import pytest

torch = pytest.importorskip("torch")

from paper_1808_01829_gb300 import functional


class FakeContext:
    made = []

    def __init__(self, dims, mass, bc_t=-1, device=0):
        self.dims, self.mass, self.bc_t, self.device = tuple(dims), mass, bc_t, device
        self.staged = 0
        self.closed = False
        FakeContext.made.append(self)

    def set_gauge(self, U):
        self.staged += 1

    def apply_mdagm_mrhs(self, X, sigma, precision, out=None):
        return ("apply", X, sigma, precision)

    def block_multishift_cg(self, B, shifts, tol, max_iter=0, precision="mixed"):
        return ("solve", list(shifts), tol, max_iter, precision)

    def close(self):
        self.closed = True


@pytest.fixture
def fake(monkeypatch):
    FakeContext.made = []
    monkeypatch.setattr(functional, "RhmcContext", FakeContext)
    functional._contexts.clear()
    yield FakeContext
    functional._contexts.clear()


def test_extents_and_context_reuse(fake):
    U = torch.zeros(6, 4, 2, 8, 4, 3, 3, dtype=torch.complex128)  # (Lt, Lz, Ly, Lx, 4, 3, 3)
    c1 = functional.context_for(U, 0.05)
    assert c1.dims == (8, 2, 4, 6) and c1.mass == 0.05 and c1.staged == 1
    assert functional.context_for(U, 0.05) is c1 and c1.staged == 1   # same tensor, unchanged
    U.add_(0.0)                                                        # in-place change
    assert functional.context_for(U, 0.05) is c1 and c1.staged == 2
    V = U.clone()                                                      # another tensor
    assert functional.context_for(V, 0.05) is c1 and c1.staged == 3
    c2 = functional.context_for(V, 0.07)                               # another mass
    assert c2 is not c1 and len(fake.made) == 2
    c3 = functional.context_for(V, 0.07, bc_t=1)                       # another boundary condition
    assert c3 is not c2 and c3.bc_t == 1
    functional.clear_contexts()
    assert c1.closed and c2.closed and c3.closed and not functional._contexts


def test_calls_forward_to_the_context(fake):
    U = torch.zeros(2, 2, 2, 2, 4, 3, 3, dtype=torch.complex128)
    X = torch.zeros(8, 3, 2, dtype=torch.complex128)
    assert functional.apply_mdagm(U, X, 0.1, sigma=0.5) == ("apply", X, 0.5, "fp64")
    assert functional.block_multishift_cg(U, X, [0.1, 0.2], 1e-8, 0.1, max_iter=7) == \
        ("solve", [0.1, 0.2], 1e-8, 7, "mixed")
    assert len(fake.made) == 1


def test_rejects_bad_link_shape(fake):
    with pytest.raises(ValueError):
        functional.context_for(torch.zeros(16, 4, 3, 3, dtype=torch.complex128), 0.1)


def test_binding_argument_checks():
    """The binding rejects host tensors, wrong dtypes, non-contiguous and misshaped
    fields before any library call."""
    from paper_1808_01829_gb300 import api

    X = torch.zeros(8, 3, 2, dtype=torch.complex128)
    with pytest.raises(ValueError, match="CUDA"):
        api._check_field(X, "X", (8, 3, 2))  # a host tensor
    if torch.cuda.is_available():  # pragma: no cover - the GPU machine
        Xd = X.cuda()
        api._check_field(Xd, "X", (8, 3, 2))
        with pytest.raises(ValueError, match="complex128"):
            api._check_field(Xd.to(torch.complex64), "X")
        with pytest.raises(ValueError, match="contiguous"):
            api._check_field(Xd.transpose(0, 1), "X")
        with pytest.raises(ValueError, match="shape"):
            api._check_field(Xd, "X", (8, 3, 3))
    assert list(api.PRECISION) == ["fp64", "mixed", "fp32", "df64"]
