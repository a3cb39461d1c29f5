"""Seeded synthetic inputs: hit points and per-iteration photons.

This module only draws inputs.  It holds none of the estimator's arithmetic
(no classification, statistics or update), so both the CUDA path and the CPU
oracle may consume what it produces.  Everything is drawn with torch on the
requested device from an explicit seed, so a scene is reproducible; the GPU
and CPU streams differ, which does not matter because the oracle always
ingests the exact arrays the GPU path used.

Scenes (the paper renders Mitsuba scenes, Sec. 6; those are not available,
so these planar scenes with known irradiance stand in for them):

* ``plane_scene``: one plane z=0, a regular grid of hit points in [0,1]^2 with
  normal +z, photons uniform on a square with flux 1/J, optionally zero flux
  for x > 0.5 (a step edge).
* ``box_scene``: the three faces z=0, y=0, x=0 of the unit box; hit points on
  a jittered grid per face; photons from a mixture of a uniform density over
  the faces and anisotropic Gaussian lobes (caustics, peak 20x the uniform
  density), with step-edge shadows (zero flux, photons still present).
  Options add RGB flux (lobe tints) and the VCM+ per-vertex pdf ratios.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

SEED_BASE = 0x5EED00

# face f: (normal axis, u axis, v axis); u x v = n for each face
_FACES = ((2, 0, 1), (1, 2, 0), (0, 1, 2))


def pack_snorm8(n: torch.Tensor) -> torch.Tensor:
    """Pack unit vectors (...,3) into uint32 words of four signed bytes
    (x, y, z, 0), each round(127 * component)."""
    q = torch.round(n.float().clamp(-1, 1) * 127).to(torch.int32) & 0xFF
    w = q[..., 0] | (q[..., 1] << 8) | (q[..., 2] << 16)
    return w.to(torch.int64).to(torch.int32).view(torch.int32)


def _gen(seed: int, stream: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed((seed * 1000003 + stream * 7919 + 12345) & 0x7FFFFFFFFFFFFFFF)
    return g


@dataclass
class HitPoints:
    pos: torch.Tensor            # (n,3) float32
    u: torch.Tensor              # (n,3) float32 tangent
    v: torch.Tensor              # (n,3) float32 bitangent
    nq: torch.Tensor | None      # (n,) int32 packed snorm8 normal, or None
    rho: torch.Tensor | None     # (n,2) float32 (rho_vm_h, rho_vc_h), VCM+
    face: torch.Tensor | None = None

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def numpy(self) -> dict:
        d = {"pos": self.pos.cpu().numpy(), "u": self.u.cpu().numpy(),
             "v": self.v.cpu().numpy()}
        if self.nq is not None:
            d["nq"] = self.nq.cpu().numpy().view("uint32")
        if self.rho is not None:
            d["rho"] = self.rho.cpu().numpy()
        return d


@dataclass
class Photons:
    pos: torch.Tensor            # (J,3) float32
    flux: torch.Tensor           # (J,) or (J,3) float32
    nq: torch.Tensor | None      # (J,) int32 packed normal, or None
    rho: torch.Tensor | None     # (J,2) float32 (rho_vm_l, rho_vc_l), VCM+
    wq: torch.Tensor | None      # (J,) int32 packed incoming direction, VCM+

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def stack_numpy(batches: list) -> dict:
    """Stack per-iteration photon batches into the oracle's (iters, J, ...)
    arrays."""
    d = {"pos": torch.stack([b.pos for b in batches]).cpu().numpy(),
         "flux": torch.stack([b.flux for b in batches]).cpu().numpy()}
    if batches[0].nq is not None:
        d["nq"] = torch.stack([b.nq for b in batches]).cpu().numpy().view("uint32")
    if batches[0].rho is not None:
        d["rho"] = torch.stack([b.rho for b in batches]).cpu().numpy()
    if batches[0].wq is not None:
        d["wq"] = torch.stack([b.wq for b in batches]).cpu().numpy().view("uint32")
    return d


# --------------------------------------------------------------------------
# single plane (tiny config, rejection-rate and unbiasedness checks)
# --------------------------------------------------------------------------
@dataclass
class PlaneScene:
    nside: int = 64
    J: int = 100_000
    r0: float = 0.02
    step: bool = True            # zero flux for x > 0.5
    lo: float = 0.0              # photon square [lo, hi]^2
    hi: float = 1.0
    seed: int = SEED_BASE

    def hitpoints(self, device="cpu") -> HitPoints:
        n = self.nside
        c = (torch.arange(n, dtype=torch.float64) + 0.5) / n
        yy, xx = torch.meshgrid(c, c, indexing="ij")
        pos = torch.stack([xx.flatten(), yy.flatten(),
                           torch.zeros(n * n, dtype=torch.float64)], 1).float()
        u = torch.tensor([1.0, 0.0, 0.0]).expand(n * n, 3).contiguous()
        v = torch.tensor([0.0, 1.0, 0.0]).expand(n * n, 3).contiguous()
        return HitPoints(pos.to(device), u.to(device), v.to(device), None, None)

    def hitpoints_jittered(self, it: int, device="cpu") -> HitPoints:
        """The hit points of iteration it traced anew through a random point
        of each pixel (SPPM-style stochastic eye paths): pixel (i, j) lands at
        ((i + a) / n, (j + b) / n, 0) with a, b uniform in [0, 1).  Same count
        and order as hitpoints(): entry h is always the same pixel."""
        n = self.nside
        g = _gen(self.seed, 100_000 + it, "cpu")
        ab = torch.rand(n * n, 2, generator=g, dtype=torch.float64)
        c = torch.arange(n, dtype=torch.float64)
        yy, xx = torch.meshgrid(c, c, indexing="ij")
        pos = torch.stack([(xx.flatten() + ab[:, 0]) / n, (yy.flatten() + ab[:, 1]) / n,
                           torch.zeros(n * n, dtype=torch.float64)], 1).float()
        u = torch.tensor([1.0, 0.0, 0.0]).expand(n * n, 3).contiguous()
        v = torch.tensor([0.0, 1.0, 0.0]).expand(n * n, 3).contiguous()
        return HitPoints(pos.to(device), u.to(device), v.to(device), None, None)

    def photons(self, it: int, device="cpu") -> Photons:
        g = _gen(self.seed, it, device)
        J = self.J
        xy = torch.rand(J, 2, generator=g, device=device, dtype=torch.float32)
        xy = self.lo + (self.hi - self.lo) * xy
        pos = torch.cat([xy, torch.zeros(J, 1, device=device)], 1).contiguous()
        flux = torch.full((J,), 1.0 / J, device=device, dtype=torch.float32)
        if self.step:
            flux = torch.where(pos[:, 0] > 0.5, torch.zeros_like(flux), flux)
        return Photons(pos, flux.contiguous(), None, None, None)

    def irradiance_density(self) -> float:
        """Photon flux per unit area on the lit part: J photons of flux 1/J
        spread over the photon square."""
        return 1.0 / (self.hi - self.lo) ** 2


# --------------------------------------------------------------------------
# three faces of the unit box with caustic lobes and shadows
# --------------------------------------------------------------------------
@dataclass
class BoxScene:
    nh: int = 1920 * 1080
    J: int = 2_000_000
    r0: float = 0.01
    n_lobes: int = 2
    n_shadows: int = 2
    lobe_peak: float = 20.0      # lobe peak density / uniform density
    rgb: bool = False
    vcm: bool = False
    seed: int = SEED_BASE + 1
    lobes: list = field(default_factory=list)
    shadows: list = field(default_factory=list)
    w_uniform: float = 1.0

    def __post_init__(self):
        g = _gen(self.seed, -1, "cpu")
        R = lambda *s: torch.rand(*s, generator=g, dtype=torch.float64)
        self.lobes = []
        for _ in range(self.n_lobes):
            face = int(torch.randint(0, 3, (1,), generator=g))
            c = 0.25 + 0.5 * R(2)
            s1, s2 = (0.005 + 0.015 * R(2)).tolist()
            th = float(R(1)) * math.pi
            tint = (0.3 + 0.7 * R(3)).tolist() if self.rgb else [1.0, 1.0, 1.0]
            self.lobes.append({"face": face, "c": c.tolist(), "s": (s1, s2),
                               "th": th, "tint": tint})
        self.shadows = []
        for k in range(self.n_shadows):
            face = int(torch.randint(0, 3, (1,), generator=g))
            if k % 2 == 0:   # half-plane through a point, random normal
                p = (0.3 + 0.4 * R(2)).tolist()
                a = float(R(1)) * 2 * math.pi
                self.shadows.append({"face": face, "kind": "half", "p": p,
                                     "n": (math.cos(a), math.sin(a))})
            else:            # axis-aligned rectangle
                lo = (0.2 + 0.4 * R(2)).tolist()
                ext = (0.1 + 0.2 * R(2)).tolist()
                self.shadows.append({"face": face, "kind": "rect", "lo": lo,
                                     "hi": [lo[0] + ext[0], lo[1] + ext[1]]})
        # lobe weight so that its peak density is lobe_peak x the uniform
        # density w_u / 3 (three unit faces)
        wl = [self.lobe_peak * (1.0 / 3.0) * 2 * math.pi * L["s"][0] * L["s"][1]
              for L in self.lobes]
        tot = 1.0 + sum(wl)
        self.w_uniform = 1.0 / tot
        for L, w in zip(self.lobes, wl):
            L["w"] = w / tot

    # -- geometry helpers -------------------------------------------------
    @staticmethod
    def _embed(face: torch.Tensor, a: torch.Tensor, b: torch.Tensor):
        """(face, a, b) face coordinates -> 3D positions, normal, u, v."""
        n = face.shape[0]
        dev = a.device
        pos = torch.zeros(n, 3, device=dev, dtype=torch.float32)
        nrm = torch.zeros(n, 3, device=dev, dtype=torch.float32)
        u = torch.zeros(n, 3, device=dev, dtype=torch.float32)
        v = torch.zeros(n, 3, device=dev, dtype=torch.float32)
        for f, (na, ua, va) in enumerate(_FACES):
            m = face == f
            pos[m, ua] = a[m]
            pos[m, va] = b[m]
            nrm[m, na] = 1.0
            u[m, ua] = 1.0
            v[m, va] = 1.0
        return pos, nrm, u, v

    def _shadowed(self, face, a, b):
        s = torch.zeros_like(a, dtype=torch.bool)
        for S in self.shadows:
            m = face == S["face"]
            if S["kind"] == "half":
                d = (a - S["p"][0]) * S["n"][0] + (b - S["p"][1]) * S["n"][1]
                s |= m & (d > 0)
            else:
                s |= (m & (a >= S["lo"][0]) & (a <= S["hi"][0])
                      & (b >= S["lo"][1]) & (b <= S["hi"][1]))
        return s

    def hitpoints(self, device="cpu") -> HitPoints:
        g = _gen(self.seed, -2, device)
        per = [self.nh // 3 + (1 if f < self.nh % 3 else 0) for f in range(3)]
        faces, As, Bs = [], [], []
        for f, nf in enumerate(per):
            nx = max(1, int(round(math.sqrt(nf * 4.0 / 3.0))))
            ny = (nf + nx - 1) // nx
            idx = torch.arange(nf, device=device)
            ix = (idx % nx).float()
            iy = (idx // nx).float()
            j = torch.rand(nf, 2, generator=g, device=device)
            As.append((ix + j[:, 0]) / nx)
            Bs.append((iy + j[:, 1]) / ny)
            faces.append(torch.full((nf,), f, device=device, dtype=torch.int64))
        face = torch.cat(faces)
        pos, nrm, u, v = self._embed(face, torch.cat(As), torch.cat(Bs))
        rho = None
        if self.vcm:
            rho = torch.exp(torch.randn(self.nh, 2, generator=g, device=device))
        return HitPoints(pos.contiguous(), u.contiguous(), v.contiguous(),
                         pack_snorm8(nrm), rho, face)

    def photons(self, it: int, device="cpu") -> Photons:
        g = _gen(self.seed, it, device)
        J = self.J
        w = torch.tensor([self.w_uniform] + [L["w"] for L in self.lobes],
                         dtype=torch.float64)
        cdf = torch.cumsum(w, 0) / w.sum()
        pick = torch.rand(J, generator=g, device=device, dtype=torch.float64)
        comp = torch.searchsorted(cdf.to(device), pick).clamp_max(len(w) - 1)
        uni = torch.rand(J, 3, generator=g, device=device, dtype=torch.float32)
        face = torch.clamp((uni[:, 0] * 3).long(), max=2)
        a = uni[:, 1].clone()
        b = uni[:, 2].clone()
        gz = torch.randn(J, 2, generator=g, device=device, dtype=torch.float32)
        tint = torch.ones(J, 3, device=device, dtype=torch.float32)
        for k, L in enumerate(self.lobes):
            m = comp == (k + 1)
            c, s = math.cos(L["th"]), math.sin(L["th"])
            x1 = gz[:, 0] * L["s"][0]
            x2 = gz[:, 1] * L["s"][1]
            a = torch.where(m, L["c"][0] + c * x1 - s * x2, a)
            b = torch.where(m, L["c"][1] + s * x1 + c * x2, b)
            face = torch.where(m, torch.full_like(face, L["face"]), face)
            tint = torch.where(m[:, None], torch.tensor(L["tint"], device=device,
                                                        dtype=torch.float32), tint)
        pos, nrm, _, _ = self._embed(face, a, b)
        lit = (~self._shadowed(face, a, b)).float()
        if self.rgb:
            flux = (tint * (lit / J)[:, None]).contiguous()
        else:
            flux = (lit / J).contiguous()
        rho = wq = None
        if self.vcm:
            rho = torch.exp(torch.randn(J, 2, generator=g, device=device))
            # cosine-distributed incoming direction around the face normal
            e = torch.rand(J, 2, generator=g, device=device)
            ct = torch.sqrt(e[:, 0])
            st = torch.sqrt(1 - e[:, 0])
            ph = 2 * math.pi * e[:, 1]
            loc = torch.stack([st * torch.cos(ph), st * torch.sin(ph), ct], 1)
            d = torch.zeros(J, 3, device=device)
            for f, (na, ua, va) in enumerate(_FACES):
                m = face == f
                d[m, ua] = loc[m, 0]
                d[m, va] = loc[m, 1]
                d[m, na] = loc[m, 2]
            wq = pack_snorm8(d)
        return Photons(pos.contiguous(), flux, pack_snorm8(nrm), rho, wq)

    def irradiance(self, hp: HitPoints) -> torch.Tensor:
        """Closed-form flux density at each hit point (the photon density per
        unit area times the photon flux J * 1/J, zero in shadows)."""
        face = hp.face
        na = torch.tensor([f[1] for f in _FACES], device=hp.pos.device)
        nb = torch.tensor([f[2] for f in _FACES], device=hp.pos.device)
        a = hp.pos.gather(1, na[face][:, None]).squeeze(1).double()
        b = hp.pos.gather(1, nb[face][:, None]).squeeze(1).double()
        dens = torch.full_like(a, self.w_uniform / 3.0)
        for L in self.lobes:
            c, s = math.cos(L["th"]), math.sin(L["th"])
            da, db = a - L["c"][0], b - L["c"][1]
            x1 = c * da + s * db
            x2 = -s * da + c * db
            gpdf = torch.exp(-0.5 * ((x1 / L["s"][0]) ** 2 + (x2 / L["s"][1]) ** 2)) \
                / (2 * math.pi * L["s"][0] * L["s"][1])
            dens = dens + torch.where(face == L["face"], L["w"] * gpdf,
                                      torch.zeros_like(gpdf))
        return dens * (~self._shadowed(face, a.float(), b.float())).double()


# --------------------------------------------------------------------------
# random-orientation unit squares (one problem of a batch)
# --------------------------------------------------------------------------
def onb_from_normal(n: torch.Tensor):
    """Tangent frame (t, b) of unit normals n (..., 3): the branchless
    construction of Duff et al., "Building an Orthonormal Basis, Revisited"
    (JCGT 2017), evaluated in float64."""
    n = n.double()
    sign = torch.where(n[..., 2] >= 0, torch.ones_like(n[..., 2]), -torch.ones_like(n[..., 2]))
    a = -1.0 / (sign + n[..., 2])
    b = n[..., 0] * n[..., 1] * a
    t = torch.stack([1.0 + sign * n[..., 0] * n[..., 0] * a, sign * b, -sign * n[..., 0]], -1)
    bb = torch.stack([b, sign + n[..., 1] * n[..., 1] * a, -n[..., 1]], -1)
    return t, bb


@dataclass
class SquaresScene:
    """1-3 unit squares with random orientation and position, hit points on a
    jittered grid per square, photons uniform over the squares plus Gaussian
    lobes (peak 20x) and step-edge shadows, flux 1/J; r0 chosen for ~150
    expected photons per disk on the uniform part."""
    nh: int = 4000
    J: int = 40_000
    n_squares: int = 2
    n_lobes: int = 2
    n_shadows: int = 2
    lobe_peak: float = 20.0
    photons_per_disk: float = 150.0
    seed: int = SEED_BASE + 2

    def __post_init__(self):
        g = _gen(self.seed, -1, "cpu")
        R = lambda *s: torch.rand(*s, generator=g, dtype=torch.float64)
        nrm = torch.randn(self.n_squares, 3, generator=g, dtype=torch.float64)
        self.normal = nrm / nrm.norm(dim=1, keepdim=True)
        self.t, self.b = onb_from_normal(self.normal)
        self.center = (R(self.n_squares, 3) - 0.5) * 3.0
        self.lobes = []
        for _ in range(self.n_lobes):
            sq = int(torch.randint(0, self.n_squares, (1,), generator=g))
            c = (0.25 + 0.5 * R(2) - 0.5).tolist()
            s1, s2 = (0.005 + 0.015 * R(2)).tolist()
            self.lobes.append({"sq": sq, "c": c, "s": (s1, s2), "th": float(R(1)) * math.pi})
        self.shadows = []
        for k in range(self.n_shadows):
            sq = int(torch.randint(0, self.n_squares, (1,), generator=g))
            if k % 2 == 0:
                p = (0.3 + 0.4 * R(2) - 0.5).tolist()
                a = float(R(1)) * 2 * math.pi
                self.shadows.append({"sq": sq, "kind": "half", "p": p, "n": (math.cos(a), math.sin(a))})
            else:
                lo = (0.2 + 0.4 * R(2) - 0.5).tolist()
                ext = (0.1 + 0.2 * R(2)).tolist()
                self.shadows.append({"sq": sq, "kind": "rect", "lo": lo,
                                     "hi": [lo[0] + ext[0], lo[1] + ext[1]]})
        area = float(self.n_squares)
        wl = [self.lobe_peak * (1.0 / area) * 2 * math.pi * L["s"][0] * L["s"][1] for L in self.lobes]
        tot = 1.0 + sum(wl)
        self.w_uniform = 1.0 / tot
        for L, w in zip(self.lobes, wl):
            L["w"] = w / tot
        self.r0 = float(math.sqrt(self.photons_per_disk * area / (math.pi * self.J)))

    def _embed(self, sq, a, b):
        c = self.center.to(a.device)[sq]
        t = self.t.to(a.device)[sq]
        bb = self.b.to(a.device)[sq]
        return (c + a.double()[:, None] * t + b.double()[:, None] * bb).float()

    def hitpoints(self, device="cpu") -> HitPoints:
        g = _gen(self.seed, -2, device)
        per = [self.nh // self.n_squares + (1 if q < self.nh % self.n_squares else 0)
               for q in range(self.n_squares)]
        sqs, As, Bs = [], [], []
        for q, nq in enumerate(per):
            nx = max(1, int(round(math.sqrt(nq))))
            ny = (nq + nx - 1) // nx
            idx = torch.arange(nq, device=device)
            j = torch.rand(nq, 2, generator=g, device=device, dtype=torch.float64)
            As.append(((idx % nx).double() + j[:, 0]) / nx - 0.5)
            Bs.append(((idx // nx).double() + j[:, 1]) / ny - 0.5)
            sqs.append(torch.full((nq,), q, device=device, dtype=torch.int64))
        sq = torch.cat(sqs)
        pos = self._embed(sq, torch.cat(As), torch.cat(Bs))
        u = self.t.to(device)[sq].float().contiguous()
        v = self.b.to(device)[sq].float().contiguous()
        nq = pack_snorm8(self.normal.to(device)[sq])
        return HitPoints(pos.contiguous(), u, v, nq, None, sq)

    def photons(self, it: int, device="cpu") -> Photons:
        g = _gen(self.seed, it, device)
        J = self.J
        w = torch.tensor([self.w_uniform] + [L["w"] for L in self.lobes], dtype=torch.float64)
        cdf = torch.cumsum(w, 0) / w.sum()
        comp = torch.searchsorted(cdf.to(device), torch.rand(J, generator=g, device=device,
                                                             dtype=torch.float64)).clamp_max(len(w) - 1)
        uni = torch.rand(J, 3, generator=g, device=device, dtype=torch.float64)
        sq = torch.clamp((uni[:, 0] * self.n_squares).long(), max=self.n_squares - 1)
        a = uni[:, 1] - 0.5
        b = uni[:, 2] - 0.5
        gz = torch.randn(J, 2, generator=g, device=device, dtype=torch.float64)
        for k, L in enumerate(self.lobes):
            m = comp == (k + 1)
            c, s_ = math.cos(L["th"]), math.sin(L["th"])
            x1, x2 = gz[:, 0] * L["s"][0], gz[:, 1] * L["s"][1]
            a = torch.where(m, L["c"][0] + c * x1 - s_ * x2, a)
            b = torch.where(m, L["c"][1] + s_ * x1 + c * x2, b)
            sq = torch.where(m, torch.full_like(sq, L["sq"]), sq)
        lit = torch.ones(J, dtype=torch.bool, device=device)
        for S in self.shadows:
            m = sq == S["sq"]
            if S["kind"] == "half":
                d = (a - S["p"][0]) * S["n"][0] + (b - S["p"][1]) * S["n"][1]
                lit &= ~(m & (d > 0))
            else:
                lit &= ~(m & (a >= S["lo"][0]) & (a <= S["hi"][0]) & (b >= S["lo"][1]) & (b <= S["hi"][1]))
        pos = self._embed(sq, a, b).contiguous()
        flux = (lit.float() / J).contiguous()
        return Photons(pos, flux, pack_snorm8(self.normal.to(device)[sq]), None, None)


def batch_scenes(n_problems=256, nh_range=(1_000, 256_000), J_range=(10_000, 1_000_000),
                 seed=SEED_BASE + 3, photons_per_disk=150.0):
    """Independent problems with log-uniform hit-point and photon counts."""
    g = _gen(seed, -3, "cpu")
    u = torch.rand(n_problems, 3, generator=g, dtype=torch.float64)
    lo_h, hi_h = math.log(nh_range[0]), math.log(nh_range[1])
    lo_j, hi_j = math.log(J_range[0]), math.log(J_range[1])
    out = []
    for p in range(n_problems):
        nh = int(round(math.exp(lo_h + (hi_h - lo_h) * float(u[p, 0]))))
        J = int(round(math.exp(lo_j + (hi_j - lo_j) * float(u[p, 1]))))
        out.append(SquaresScene(nh=nh, J=J, n_squares=1 + int(float(u[p, 2]) * 3),
                                photons_per_disk=photons_per_disk, seed=seed + 17 * (p + 1)))
    return out
