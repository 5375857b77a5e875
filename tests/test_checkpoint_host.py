"""Training-checkpoint files (precond.save_checkpoint / load_checkpoint) on
the host: weights, Adam moments, the step count and extra scalars survive the
.npz round trip exactly, and the restore order is weights first (which resets
Adam in the library), then the Adam state.  A stand-in object with the
network's accessor methods replaces the device network."""
import numpy as np

from paper_1604_03155_gb300 import precond as P


class _Net:
    def __init__(self, n, seed):
        rng = np.random.default_rng(seed)
        self.w = rng.standard_normal(n).astype(np.float32)
        self.m = rng.standard_normal(n).astype(np.float32)
        self.v = rng.random(n).astype(np.float32)
        self.step = int(rng.integers(1, 1000))
        self.calls = []

    def get(self, which=0):
        assert which == 0
        return self.w.copy()

    def get_adam(self):
        return self.m.copy(), self.v.copy(), self.step

    def set_weights(self, w):
        self.calls.append("weights")
        self.w = np.asarray(w, np.float32).copy()
        self.m[:] = 0
        self.v[:] = 0
        self.step = 0

    def set_adam(self, m, v, step):
        self.calls.append("adam")
        self.m, self.v, self.step = np.asarray(m).copy(), np.asarray(v).copy(), int(step)


def test_checkpoint_round_trip(tmp_path):
    a = _Net(1234, 1)
    path = str(tmp_path / "ck.npz")
    P.save_checkpoint(a, path, next_contrast=17, lr=3e-3)
    b = _Net(1234, 2)
    extra = P.load_checkpoint(b, path)
    assert b.calls == ["weights", "adam"]
    assert np.array_equal(a.w, b.w) and np.array_equal(a.m, b.m) and np.array_equal(a.v, b.v)
    assert b.step == a.step
    assert extra == {"next_contrast": 17, "lr": 3e-3}
