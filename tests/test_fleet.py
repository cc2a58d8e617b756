"""The fleet load generator (host logic, no device): a controller per
environment ticking at a fixed rate, skipped ticks counted while a request
is pending, Poisson resets passed to the server, nothing lost.  A fake
server with a simulated clock stands in for BatchServer: it answers each
request a fixed latency after submission, at most `cap` per step."""
import numpy as np

from paper_2606_05687_b300.serve import fleet_load


class FakeServer:
    def __init__(self, n_env, latency, dt=1e-3, cap=None):
        self.pool = {"A": np.zeros((n_env, 1))}
        self.latency, self.dt, self.cap = latency, dt, cap
        self.t = 0.0
        size = 1 << 20
        self.env = np.zeros(size, np.int64)
        self.t_arrival = np.zeros(size)
        self.t_sub = np.zeros(size)
        self.t_done = np.full(size, np.nan)
        self.status = np.full(size, -1, np.int32)
        self.n = 0
        self.head = 0  # first unanswered request (answers are first-in first-out)
        self.reset_envs = []

    def clock(self):
        return self.t

    def submit(self, envs, t_arrival):
        k = len(envs)
        self.env[self.n:self.n + k] = envs
        self.t_arrival[self.n:self.n + k] = t_arrival
        self.t_sub[self.n:self.n + k] = self.t
        self.n += k

    def reset(self, envs):
        self.reset_envs.extend(int(e) for e in envs)

    def step(self):
        self.t += self.dt
        served = 0
        while self.head < self.n and self.t_sub[self.head] + self.latency <= self.t:
            if self.cap is not None and served >= self.cap:
                break
            self.t_done[self.head] = self.t
            self.status[self.head] = 0
            self.head += 1
            served += 1

    def drain(self):
        while self.head < self.n:
            self.step()


def test_every_tick_requests_when_answers_come_in_time():
    srv = FakeServer(n_env=100, latency=0.005)
    r = fleet_load(srv, hz=50.0, duration=1.0, seed=1)
    assert r["skipped_ticks"] == 0
    assert abs(r["offered_ticks_per_s"] - 100 * 50) <= 100
    assert r["requests"] == r["offered_ticks_per_s"] * 1.0
    assert r["certified"] == r["requests"]
    # tick to answer: the latency plus at most two clock steps of looking late
    assert 5.0 <= r["p50_ms"] <= 7.5 and r["p99_ms"] <= 7.5
    assert np.all(np.isfinite(srv.t_done[:srv.n]))
    # each environment has at most one request in flight
    for e in (0, 17, 99):
        req = np.flatnonzero(srv.env[:srv.n] == e)
        assert np.all(srv.t_arrival[req[1:]] >= srv.t_done[req[:-1]] - 1e-12)


def test_overload_skips_ticks_and_serves_at_capacity():
    # 5000 ticks/s offered, 1000 answers/s of capacity
    srv = FakeServer(n_env=100, latency=0.0, cap=1)
    r = fleet_load(srv, hz=50.0, duration=2.0, seed=2)
    ticks = r["offered_ticks_per_s"] * 2.0
    assert ticks - r["skipped_ticks"] == r["requests"]  # every tick is a request or counted as skipped
    assert r["skipped_ticks"] > 0.7 * ticks
    assert abs(r["answered_per_s"] - 1000) <= 20
    assert np.all(np.isfinite(srv.t_done[:srv.n]))  # nothing lost


def test_resets_reach_the_server_at_the_poisson_rate():
    srv = FakeServer(n_env=1000, latency=0.002, dt=2e-3)
    r = fleet_load(srv, hz=10.0, duration=2.0, reset_rate=0.5, seed=3)
    assert r["resets"] == len(srv.reset_envs)
    assert abs(r["resets"] - 1000) <= 4 * np.sqrt(1000)
    assert len(set(srv.reset_envs)) > 500


def test_warmup_window_excludes_early_requests():
    srv = FakeServer(n_env=50, latency=0.001)
    r = fleet_load(srv, hz=20.0, duration=1.0, warmup=0.5, seed=4)
    assert abs(r["requests"] - 50 * 20) <= 50
    assert srv.n > r["requests"]  # the warm-up's requests were served but are not counted
